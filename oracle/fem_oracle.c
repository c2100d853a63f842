/*
 * fem_oracle.c -- plain, slow FP64 CPU oracle for per-element numerical
 * integration (Banas, Plaszewski, Maciol, "Numerical integration on GPUs for
 * higher order finite elements", arXiv 1310.1191).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code.  It shares no source with the
 * CUDA library: quadrature comes from Newton iteration on Jacobi polynomials
 * (the library uses Golub-Welsch), Jacobi polynomials come from their explicit
 * finite sum (the library uses the three-term recurrence), and the element
 * map derivatives come from the six vertex shape functions (the library uses
 * edge vectors).
 *
 * What it computes (Section 2, eq. sum_int): the quadrature sum of the weak
 * form over each element, written out as its definition:
 *   phi_Q[iD][i]  reference shape functions (iD=0) and their reference
 *                 derivatives (iD=1..3) at quadrature point Q,
 *   J_Q, det J_Q, J_Q^{-1}  Jacobian of the reference->real map,
 *   psi_Q[iD][i]  physical table by the chain rule:
 *                 d phi/d x_m = sum_k d phi/d xi_k * (J^{-1})[k][m],
 *   C_Q[iD][jD]   4x4 coefficient matrix of the form at the point,
 *   A^e = sum_Q w_Q det J_Q psi_Q^T C_Q psi_Q.
 * The generic second-order form is -div(D grad u) + b.grad u + c u = f, i.e.
 *   C[0][0] = c, C[0][1+m] = b_m, C[1+l][1+m] = D[l][m], C[1+l][0] = 0,
 * row i = test function, column j = trial function.  The load vector (not in
 * the paper, which integrates only A^e) is b^e[i] = sum_Q w det f psi[0][i].
 *
 * Readings where the paper is silent (it names a prism with complete
 * triangle polynomials times 1D polynomials and "Gaussian" quadrature,
 * Section 2, Table 1):
 *   - reference prism {xi,eta >= 0, xi+eta <= 1} x zeta in [-1,1], vertices
 *     0..2 at zeta=-1 ((0,0),(1,0),(0,1)), 3..5 above them at zeta=+1;
 *   - basis: Dubiner triangle functions in collapsed coordinates
 *     (r=2xi-1, s=2eta-1, a=2(1+r)/(1-s)-1, b=s)
 *       psi_ij = P_i^(0,0)(a) ((1-b)/2)^i P_j^(2i+1,0)(b), i+j <= p,
 *     unnormalised, times Legendre L_k(zeta), k <= p; DOF index t + NT*k with
 *     t running over n=i+j ascending, then i descending;
 *   - quadrature: (p+1) points per direction, Gauss-Legendre in a,
 *     Gauss-Jacobi(1,0) in b, Gauss-Legendre in zeta; xi=(1+a)(1-b)/4,
 *     eta=(1+b)/2, w = wa wb wz / 8; point order q = iz*n*n + ia*n + ib;
 *   - tetrahedron: P1 basis (barycentric), textbook 4-point degree-2 rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TET 0
#define ORC_PRISM 1
#define ORC_PRISM_T1 2 /* prism with the paper's rule (Table 1 point counts) */

#define ORC_ST_DET 1      /* det J <= 0 at some quadrature point */
#define ORC_ST_NONFINITE 2 /* non-finite geometry or coefficient input */
#define ORC_ST_FALLBACK 8  /* surrogate input outside its box: exact law used */

typedef long double ld;

/* ------------------------------------------------------------------ sizes */
int orc_ns(int elem, int p) {
    if (elem == ORC_TET) return p == 1 ? 4 : -1;
    if ((elem != ORC_PRISM && elem != ORC_PRISM_T1) || p < 1 || p > 7) return -1;
    return (p + 1) * (p + 1) * (p + 2) / 2;
}

static const int orc_tri_count[8] = {0, 3, 6, 12, 16, 25, 33, 42};

int orc_nq(int elem, int p) {
    if (elem == ORC_TET) return p == 1 ? 4 : -1;
    if ((elem != ORC_PRISM && elem != ORC_PRISM_T1) || p < 1 || p > 7) return -1;
    if (elem == ORC_PRISM_T1) return (p + 1) * orc_tri_count[p];
    return (p + 1) * (p + 1) * (p + 1);
}

/* -------------------------------------------------- Jacobi polynomials */
static ld binom_l(int n, int k) {
    if (k < 0 || k > n) return 0.0L;
    ld r = 1.0L;
    for (int i = 1; i <= k; i++) r = r * (ld)(n - k + i) / (ld)i;
    return r;
}

static ld ipow_l(ld x, int k) {
    ld r = 1.0L;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

/* P_n^(a,b)(x) by its explicit finite sum
 *   sum_s C(n+a, n-s) C(n+b, s) ((x-1)/2)^s ((x+1)/2)^(n-s). */
static ld jacobi_l(int n, int a, int b, ld x) {
    if (n < 0) return 0.0L;
    ld xm = (x - 1.0L) / 2.0L, xp = (x + 1.0L) / 2.0L, s = 0.0L;
    for (int k = 0; k <= n; k++)
        s += binom_l(n + a, n - k) * binom_l(n + b, k) * ipow_l(xm, k) * ipow_l(xp, n - k);
    return s;
}

/* d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1) */
static ld djacobi_l(int n, int a, int b, ld x) {
    if (n <= 0) return 0.0L;
    return 0.5L * (ld)(n + a + b + 1) * jacobi_l(n - 1, a + 1, b + 1, x);
}

double orc_jacobi(int n, int a, int b, double x) { return (double)jacobi_l(n, a, b, x); }
double orc_djacobi(int n, int a, int b, double x) { return (double)djacobi_l(n, a, b, x); }

/* ---------------------------------------------- Gauss-Jacobi quadrature */
/* Roots of P_n^(a,b) by Newton's method with deflation of the roots already
 * found (Chebyshev points as first guesses), weights from
 *   w_k = 2^(a+b+1) G(n+a+1) G(n+b+1) / (G(n+a+b+1) n!) / ((1-x_k^2) P_n'(x_k)^2).
 * Nodes ascending.  Exact for polynomials of degree <= 2n-1 against
 * (1-x)^a (1+x)^b on [-1,1]. */
void orc_gauss_jacobi(int n, int a, int b, double *x, double *w) {
    ld r[16];
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < n; k++) {
        ld z = -cosl((2.0L * k + 1.0L) * pi / (2.0L * n));
        if (k > 0) z = 0.5L * (z + r[k - 1]);
        for (int it = 0; it < 200; it++) {
            ld f = jacobi_l(n, a, b, z), fp = djacobi_l(n, a, b, z), s = 0.0L;
            for (int i = 0; i < k; i++) s += 1.0L / (z - r[i]);
            ld dz = -f / (fp - s * f);
            z += dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        r[k] = z;
    }
    ld c = powl(2.0L, (ld)(a + b + 1)) * tgammal((ld)(n + a + 1)) * tgammal((ld)(n + b + 1)) /
           (tgammal((ld)(n + a + b + 1)) * tgammal((ld)(n + 1)));
    for (int k = 0; k < n; k++) {
        ld d = djacobi_l(n, a, b, r[k]);
        x[k] = (double)r[k];
        w[k] = (double)(c / ((1.0L - r[k] * r[k]) * d * d));
    }
}

int orc_tri_rule(int p, double *x, double *y, double *w);

/* Quadrature rule on the reference element; returns NQ or -1.
 * xi: [NQ][3], w: [NQ]. */
int orc_rule(int elem, int p, double *xi, double *w) {
    if (elem == ORC_TET) {
        if (p != 1) return -1;
        /* barycentric (al, be, be, be) and permutations, weights 1/24 (volume 1/6) */
        ld al = (5.0L + 3.0L * sqrtl(5.0L)) / 20.0L, be = (5.0L - sqrtl(5.0L)) / 20.0L;
        ld pts[4][3] = {{be, be, be}, {al, be, be}, {be, al, be}, {be, be, al}};
        for (int q = 0; q < 4; q++) {
            for (int k = 0; k < 3; k++) xi[3 * q + k] = (double)pts[q][k];
            w[q] = (double)(1.0L / 24.0L);
        }
        return 4;
    }
    if (orc_nq(elem, p) < 0) return -1;
    int n = p + 1;
    double xa[16], wa[16], xb[16], wb[16];
    orc_gauss_jacobi(n, 0, 0, xa, wa);
    orc_gauss_jacobi(n, 1, 0, xb, wb);
    if (elem == ORC_PRISM_T1) {
        /* symmetric triangle rule x Gauss-Legendre: point q = iz * NT + it */
        double tx[64], ty[64], tw[64];
        int nt = orc_tri_rule(p, tx, ty, tw);
        if (nt < 0) return -1;
        for (int iz = 0; iz < n; iz++)
            for (int it = 0; it < nt; it++) {
                int q = iz * nt + it;
                xi[3 * q + 0] = tx[it];
                xi[3 * q + 1] = ty[it];
                xi[3 * q + 2] = xa[iz];
                w[q] = tw[it] * wa[iz];
            }
        return n * nt;
    }
    int q = 0;
    for (int iz = 0; iz < n; iz++)
        for (int ia = 0; ia < n; ia++)
            for (int ib = 0; ib < n; ib++, q++) {
                xi[3 * q + 0] = (1.0 + xa[ia]) * (1.0 - xb[ib]) / 4.0;
                xi[3 * q + 1] = (1.0 + xb[ib]) / 2.0;
                xi[3 * q + 2] = xa[iz];
                w[q] = wa[ia] * wb[ib] * wa[iz] / 8.0;
            }
    return q;
}

/* ---------------------------------------- the paper's prism rules (Table 1) */
/* Table 1 gives N_Q = 6, 18, 48, 80, 150, 231, 336 = (p + 1) x (3, 6, 12, 16,
 * 25, 33, 42): a fully symmetric degree-2p triangle rule times (p + 1)-point
 * Gauss-Legendre in zeta (the paper calls them Gaussian; the triangle rules
 * are not printed).  Reading: with n0 centroids, n1 orbits (a, a, 1-2a) and n2
 * orbits (a, b, 1-a-b) in barycentric coordinates, the point count and a
 * square moment system fix (n0, n1, n2) = (0,1,0), (0,2,0), (0,2,1), (1,3,1),
 * (1,2,3), (0,5,3), (0,6,4); the rule is the positive-interior solution of the
 * moment equations, the one with the largest smallest barycentric coordinate
 * where several exist.
 *
 * orc_tri_search finds the positive-interior solutions: from random starts,
 * homotopy continuation that moves the target moments linearly from the
 * start's own moments to the exact ones; the moments are those of every
 * monomial xi^i eta^j, i + j <= 2p (closed form i! j! / (i + j + 2)!), an
 * overdetermined but consistent system solved by Gauss-Newton steps; points
 * stay strictly inside and weights positive through the parameters
 * a = 1 / (2 (1 + e^-s)) (S21), (a, b, c) = softmax(s1, s2, 0) (S111),
 * w = e^t.  Each solution is polished in long double and stored in canonical
 * order (S21 by a; S111 as a < b < c, by (a, b)). */
static const int orc_tri_shape[8][3] = {{0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 2, 1},
                                        {1, 3, 1}, {1, 2, 3}, {0, 5, 3}, {0, 6, 4}};

int orc_tri_points(int p) {
    if (p < 1 || p > 7) return -1;
    return orc_tri_shape[p][0] + 3 * orc_tri_shape[p][1] + 6 * orc_tri_shape[p][2];
}

int orc_tri_unknowns(int p) {
    if (p < 1 || p > 7) return -1;
    return orc_tri_shape[p][0] + 2 * orc_tri_shape[p][1] + 3 * orc_tri_shape[p][2];
}

/* barycentric points (l0, l1, l2) and weights of the orbits with natural
 * parameters x (centroid w; S21 a, w; S111 a, b, w) */
static int tri_expand(int p, const ld *x, ld (*l)[3], ld *w) {
    int n = 0, k = 0;
    for (int o = 0; o < orc_tri_shape[p][0]; o++, k++) {
        l[n][0] = l[n][1] = l[n][2] = 1.0L / 3.0L;
        w[n++] = x[k];
    }
    for (int o = 0; o < orc_tri_shape[p][1]; o++, k += 2) {
        ld a = x[k], c = 1.0L - 2.0L * a;
        ld pts[3][3] = {{a, a, c}, {a, c, a}, {c, a, a}};
        for (int m = 0; m < 3; m++, n++) {
            for (int d = 0; d < 3; d++) l[n][d] = pts[m][d];
            w[n] = x[k + 1];
        }
    }
    for (int o = 0; o < orc_tri_shape[p][2]; o++, k += 3) {
        ld a = x[k], b = x[k + 1], c = 1.0L - a - b;
        ld pts[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
        for (int m = 0; m < 6; m++, n++) {
            for (int d = 0; d < 3; d++) l[n][d] = pts[m][d];
            w[n] = x[k + 2];
        }
    }
    return n;
}

/* exact monomial moments of the triangle, i! j! / (i + j + 2)!, i + j <= 2p */
static void tri_exact(int p, double *ex) {
    int m = 0;
    for (int i = 0; i <= 2 * p; i++)
        for (int j = 0; i + j <= 2 * p; j++, m++)
            ex[m] = (double)(tgammal(i + 1) * tgammal(j + 1) / tgammal(i + j + 3));
}

/* natural parameters x from the free parameters z, and dx/dz (block diagonal:
 * per orbit), see the search's description above */
static void tri_natural(int p, const double *z, double *x, double (*dx)[40]) {
    const int nu = orc_tri_unknowns(p);
    for (int a = 0; a < nu; a++)
        for (int b = 0; b < nu; b++) dx[a][b] = 0.0;
    int k = 0;
    for (int o = 0; o < orc_tri_shape[p][0]; o++, k++) x[k] = dx[k][k] = exp(z[k]);
    for (int o = 0; o < orc_tri_shape[p][1]; o++, k += 2) {
        double sg = 1.0 / (1.0 + exp(-z[k]));
        x[k] = 0.5 * sg;
        dx[k][k] = 0.5 * sg * (1.0 - sg);
        x[k + 1] = dx[k + 1][k + 1] = exp(z[k + 1]);
    }
    for (int o = 0; o < orc_tri_shape[p][2]; o++, k += 3) {
        double m = z[k] > z[k + 1] ? z[k] : z[k + 1];
        m = m > 0.0 ? m : 0.0;
        double e1 = exp(z[k] - m), e2 = exp(z[k + 1] - m), Z = e1 + e2 + exp(-m);
        double a = e1 / Z, b = e2 / Z;
        x[k] = a;
        x[k + 1] = b;
        dx[k][k] = a * (1.0 - a);
        dx[k][k + 1] = -a * b;
        dx[k + 1][k] = -a * b;
        dx[k + 1][k + 1] = b * (1.0 - b);
        x[k + 2] = dx[k + 2][k + 2] = exp(z[k + 2]);
    }
}

/* moments (over the exact ones) of the rule with natural parameters x, and
 * their derivatives d mom / d x (analytic) */
static int tri_moments_d(int p, const double *x, const double *ex, double *mom, double (*J)[40]) {
    const int nm = (2 * p + 1) * (2 * p + 2) / 2, nu = orc_tri_unknowns(p), d = 2 * p;
    for (int m = 0; m < nm; m++) {
        mom[m] = 0.0;
        for (int a = 0; a < nu; a++) J[m][a] = 0.0;
    }
    /* TRI_POINT: one point (l1, l2) = (xi, eta) of weight w, Jacobian
     * columns cw (its weight) and c0.. (its np position parameters, with
     * d l1 / d param = d1[], d l2 / d param = d2[]) */
    int k = 0;
#define TRI_POINT(L1, L2, W, CW, C0, NP, D1, D2)                                                  \
    do {                                                                                          \
        double p1[16], p2[16];                                                                    \
        p1[0] = p2[0] = 1.0;                                                                      \
        for (int e = 1; e <= d; e++) {                                                            \
            p1[e] = p1[e - 1] * (L1);                                                             \
            p2[e] = p2[e - 1] * (L2);                                                             \
        }                                                                                         \
        int m_ = 0;                                                                               \
        for (int i = 0; i <= d; i++)                                                              \
            for (int j = 0; i + j <= d; j++, m_++) {                                              \
                double v = p1[i] * p2[j] / ex[m_];                                                \
                double g1 = i ? i * p1[i - 1] * p2[j] / ex[m_] : 0.0;                             \
                double g2 = j ? j * p1[i] * p2[j - 1] / ex[m_] : 0.0;                             \
                mom[m_] += (W) * v;                                                               \
                J[m_][CW] += v;                                                                   \
                for (int q_ = 0; q_ < (NP); q_++) J[m_][(C0) + q_] += (W) * (g1 * (D1)[q_] + g2 * (D2)[q_]); \
            }                                                                                     \
    } while (0)
    for (int o = 0; o < orc_tri_shape[p][0]; o++, k++) {
        const double z0[1] = {0.0};
        TRI_POINT(1.0 / 3.0, 1.0 / 3.0, x[k], k, k, 0, z0, z0);
    }
    for (int o = 0; o < orc_tri_shape[p][1]; o++, k += 2) {
        double a = x[k], c = 1.0 - 2.0 * a, w = x[k + 1];
        /* (l1, l2) = (a, c), (c, a), (a, a); d/da */
        const double da1[3] = {1.0, -2.0, 1.0}, da2[3] = {-2.0, 1.0, 1.0};
        const double l1[3] = {a, c, a}, l2[3] = {c, a, a};
        for (int m = 0; m < 3; m++) TRI_POINT(l1[m], l2[m], w, k + 1, k, 1, &da1[m], &da2[m]);
    }
    for (int o = 0; o < orc_tri_shape[p][2]; o++, k += 3) {
        double a = x[k], b = x[k + 1], c = 1.0 - a - b, w = x[k + 2];
        /* the six permutations (l0, l1, l2) of (a, b, c); (l1, l2) and d/d(a, b) */
        const double l1[6] = {b, c, a, c, a, b}, l2[6] = {c, b, c, a, b, a};
        const double d1[6][2] = {{0, 1}, {-1, -1}, {1, 0}, {-1, -1}, {1, 0}, {0, 1}};
        const double d2[6][2] = {{-1, -1}, {0, 1}, {-1, -1}, {1, 0}, {0, 1}, {1, 0}};
        for (int m = 0; m < 6; m++) TRI_POINT(l1[m], l2[m], w, k + 2, k, 2, d1[m], d2[m]);
    }
#undef TRI_POINT
    return nm;
}

/* Gauss-Newton step: (J^T J) dz = -J^T r; 0 if singular */
static int tri_gn_step(int nu, int nm, double (*J)[40], const double *r, double *dz) {
    double A[40][41];
    for (int a = 0; a < nu; a++) {
        for (int b = 0; b < nu; b++) {
            double s = 0.0;
            for (int m = 0; m < nm; m++) s += J[m][a] * J[m][b];
            A[a][b] = s;
        }
        double s = 0.0;
        for (int m = 0; m < nm; m++) s -= J[m][a] * r[m];
        A[a][nu] = s;
    }
    for (int c = 0; c < nu; c++) {
        int pv = c;
        for (int q = c + 1; q < nu; q++)
            if (fabs(A[q][c]) > fabs(A[pv][c])) pv = q;
        if (!(fabs(A[pv][c]) > 1e-300)) return 0;
        for (int q = 0; q <= nu; q++) {
            double t = A[c][q];
            A[c][q] = A[pv][q];
            A[pv][q] = t;
        }
        for (int q = c + 1; q < nu; q++) {
            double f = A[q][c] / A[c][c];
            for (int k = c; k <= nu; k++) A[q][k] -= f * A[c][k];
        }
    }
    for (int q = nu - 1; q >= 0; q--) {
        double s = A[q][nu];
        for (int k = q + 1; k < nu; k++) s -= A[q][k] * dz[k];
        dz[q] = s / A[q][q];
    }
    return 1;
}

static uint64_t orc_splitmix(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double orc_unif(uint64_t *s) { return (double)(orc_splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

/* one continuation path from a seeded start; 1 and the natural parameters x on success */
static int tri_path(int p, uint64_t seed, const double *ex, double *x) {
    const int nu = orc_tri_unknowns(p), npt = orc_tri_points(p), nm = (2 * p + 1) * (2 * p + 2) / 2;
    double z[40], m0[200], mom[200], r[200], Jx[200][40], Jz[200][40], dxz[40][40];
    int k = 0;
    for (int o = 0; o < orc_tri_shape[p][0]; o++) z[k++] = log(0.5 / npt) + 0.6 * (orc_unif(&seed) - 0.5);
    for (int o = 0; o < orc_tri_shape[p][1]; o++) {
        z[k++] = 6.0 * (orc_unif(&seed) - 0.5);
        z[k++] = log(0.5 / npt) + 0.6 * (orc_unif(&seed) - 0.5);
    }
    for (int o = 0; o < orc_tri_shape[p][2]; o++) {
        z[k++] = 5.0 * (orc_unif(&seed) - 0.5);
        z[k++] = 5.0 * (orc_unif(&seed) - 0.5);
        z[k++] = log(0.5 / npt) + 0.6 * (orc_unif(&seed) - 0.5);
    }
    tri_natural(p, z, x, dxz);
    tri_moments_d(p, x, ex, m0, Jx);
    double t = 0.0, dt = 0.02;
    while (t < 1.0) {
        double tn = t + dt > 1.0 ? 1.0 : t + dt, z2[40];
        memcpy(z2, z, sizeof(double) * nu);
        int good = 0;
        for (int it = 0; it < 6; it++) {
            tri_natural(p, z2, x, dxz);
            tri_moments_d(p, x, ex, mom, Jx);
            double nr = 0.0;
            for (int m = 0; m < nm; m++) {
                r[m] = mom[m] - ((1.0 - tn) * m0[m] + tn);
                nr = fabs(r[m]) > nr ? fabs(r[m]) : nr;
                for (int a = 0; a < nu; a++) {  /* chain rule through dx/dz */
                    double s = 0.0;
                    for (int b = 0; b < nu; b++) s += Jx[m][b] * dxz[b][a];
                    Jz[m][a] = s;
                }
            }
            if (!(nr == nr)) break;
            if (nr < 1e-11) {
                good = 1;
                break;
            }
            double dz[40], mx = 0.0;
            if (!tri_gn_step(nu, nm, Jz, r, dz)) break;
            for (int a = 0; a < nu; a++) mx = fabs(dz[a]) > mx ? fabs(dz[a]) : mx;
            if (mx > 2.0) break;
            for (int a = 0; a < nu; a++) z2[a] += dz[a];
        }
        double mz = 0.0;
        for (int a = 0; a < nu; a++) mz = fabs(z2[a]) > mz ? fabs(z2[a]) : mz;
        if (good && mz < 40.0) {
            memcpy(z, z2, sizeof(double) * nu);
            t = tn;
            dt = dt * 1.3 > 0.05 ? 0.05 : dt * 1.3;
        } else {
            dt *= 0.5;
            if (dt < 1e-6) return 0;
        }
    }
    tri_natural(p, z, x, dxz);
    return 1;
}

/* exactness residual of the rule in long double: max over the monomials of
 * |sum_q w_q xi^i eta^j / exact - 1| */
static ld tri_residual_l(int p, const ld *x, ld *r) {
    ld l[64][3], w[64], nr = 0.0L;
    int n = tri_expand(p, x, l, w), m = 0;
    for (int i = 0; i <= 2 * p; i++)
        for (int j = 0; i + j <= 2 * p; j++, m++) {
            ld ex = tgammal(i + 1) * tgammal(j + 1) / tgammal(i + j + 3), s = 0.0L;
            for (int q = 0; q < n; q++) s += w[q] * ipow_l(l[q][1], i) * ipow_l(l[q][2], j);
            r[m] = s / ex - 1.0L;
            nr = fabsl(r[m]) > nr ? fabsl(r[m]) : nr;
        }
    return nr;
}

/* Gauss-Newton polish in the natural parameters: residual in long double,
 * Jacobian in double (iterative refinement); 1 if it drops below 1e-17 */
static int tri_polish(int p, const double *ex, ld *x) {
    const int nu = orc_tri_unknowns(p), nm = (2 * p + 1) * (2 * p + 2) / 2;
    ld rl[200];
    double xd[40], mom[200], J[200][40], r[200], dx[40];
    for (int it = 0; it < 10; it++) {
        if (tri_residual_l(p, x, rl) < 1e-17L) return 1;
        for (int a = 0; a < nu; a++) xd[a] = (double)x[a];
        tri_moments_d(p, xd, ex, mom, J);
        for (int m = 0; m < nm; m++) r[m] = (double)rl[m];
        if (!tri_gn_step(nu, nm, J, r, dx)) return 0;
        for (int a = 0; a < nu; a++) x[a] += (ld)dx[a];
    }
    return tri_residual_l(p, x, rl) < 1e-17L;
}

static void tri_canonical(int p, ld *x) {
    int k = orc_tri_shape[p][0];
    int n1 = orc_tri_shape[p][1], n2 = orc_tri_shape[p][2];
    for (int i = 0; i < n1; i++)  /* S21 by a: insertion sort of (a, w) pairs */
        for (int j = i + 1; j < n1; j++)
            if (x[k + 2 * j] < x[k + 2 * i]) {
                ld ta = x[k + 2 * i], tw = x[k + 2 * i + 1];
                x[k + 2 * i] = x[k + 2 * j];
                x[k + 2 * i + 1] = x[k + 2 * j + 1];
                x[k + 2 * j] = ta;
                x[k + 2 * j + 1] = tw;
            }
    k += 2 * n1;
    for (int o = 0; o < n2; o++) {  /* a < b < c within each S111 orbit */
        ld v[3] = {x[k + 3 * o], x[k + 3 * o + 1], 1.0L - x[k + 3 * o] - x[k + 3 * o + 1]};
        for (int i = 0; i < 3; i++)
            for (int j = i + 1; j < 3; j++)
                if (v[j] < v[i]) {
                    ld t = v[i];
                    v[i] = v[j];
                    v[j] = t;
                }
        x[k + 3 * o] = v[0];
        x[k + 3 * o + 1] = v[1];
    }
    for (int i = 0; i < n2; i++)  /* S111 orbits by (a, b) */
        for (int j = i + 1; j < n2; j++) {
            ld *u = x + k + 3 * i, *v = x + k + 3 * j;
            if (v[0] < u[0] || (v[0] == u[0] && v[1] < u[1]))
                for (int q = 0; q < 3; q++) {
                    ld t = u[q];
                    u[q] = v[q];
                    v[q] = t;
                }
        }
}

static ld tri_min_bary(int p, const ld *x) {
    ld l[64][3], w[64], mb = 1.0L;
    int n = tri_expand(p, x, l, w);
    for (int q = 0; q < n; q++)
        for (int d = 0; d < 3; d++) mb = l[q][d] < mb ? l[q][d] : mb;
    return mb;
}

/* Runs `trials` seeded paths for degree 2p; stores up to max_sol distinct
 * positive-interior solutions (natural parameters, canonical order, sorted by
 * smallest barycentric coordinate, largest first) in sol[max_sol][unknowns]
 * and that coordinate in minb[]; returns the number stored, -1 on bad input. */
int orc_tri_search(int p, int64_t trials, uint64_t seed, int max_sol, double *sol, double *minb) {
    const int nu = orc_tri_unknowns(p);
    if (nu < 0 || max_sol < 1 || trials < 1) return -1;
    ld *found = (ld *)malloc(sizeof(ld) * 40 * (size_t)max_sol);
    int nfound = 0;
    double ex[200];
    tri_exact(p, ex);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t tr = 0; tr < trials; tr++) {
        ld x[40];
        double xd[40];
        uint64_t s = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(tr + 1));
        orc_splitmix(&s);
        if (!tri_path(p, s, ex, xd)) continue;
        for (int a = 0; a < nu; a++) x[a] = xd[a];
        if (!tri_polish(p, ex, x)) continue;
        tri_canonical(p, x);
        ld l[64][3], w[64];
        int n = tri_expand(p, x, l, w), ok = tri_min_bary(p, x) > 1e-9L;
        for (int q = 0; q < n; q++) ok = ok && w[q] > 0.0L;
        if (!ok) continue;
#pragma omp critical
        {
            int dup = 0;
            for (int f = 0; f < nfound && !dup; f++) {
                ld d = 0.0L;
                for (int a = 0; a < nu; a++) d = fabsl(found[40 * f + a] - x[a]) > d ? fabsl(found[40 * f + a] - x[a]) : d;
                dup = d < 1e-10L;
            }
            if (!dup && nfound < max_sol) {
                memcpy(found + 40 * nfound, x, sizeof(ld) * nu);
                nfound++;
            }
        }
    }
    /* sort by smallest barycentric coordinate, largest first */
    for (int i = 0; i < nfound; i++)
        for (int j = i + 1; j < nfound; j++)
            if (tri_min_bary(p, found + 40 * j) > tri_min_bary(p, found + 40 * i))
                for (int a = 0; a < 40; a++) {
                    ld t = found[40 * i + a];
                    found[40 * i + a] = found[40 * j + a];
                    found[40 * j + a] = t;
                }
    for (int f = 0; f < nfound; f++) {
        for (int a = 0; a < nu; a++) sol[(size_t)f * nu + a] = (double)found[40 * f + a];
        minb[f] = (double)tri_min_bary(p, found + 40 * f);
    }
    free(found);
    return nfound;
}

/* The triangle rules the oracle uses for the Table 1 prism rules, set once
 * from the stored result of orc_tri_search (oracle/prism_rules_table1.txt). */
static double orc_tri_params[8][40];
static int orc_tri_set[8];

int orc_set_tri_rule(int p, const double *params) {
    if (p < 1 || p > 7) return -1;
    memcpy(orc_tri_params[p], params, sizeof(double) * orc_tri_unknowns(p));
    orc_tri_set[p] = 1;
    return 0;
}

/* Points (xi, eta) = (l1, l2) and weights of the stored triangle rule of
 * degree 2p (the orbits expanded as in tri_expand); returns the number of
 * points, -1 if no rule is set for p. */
int orc_tri_rule(int p, double *x, double *y, double *w) {
    if (p < 1 || p > 7 || !orc_tri_set[p]) return -1;
    ld xp[40], l[64][3], wl[64];
    for (int a = 0; a < orc_tri_unknowns(p); a++) xp[a] = orc_tri_params[p][a];
    int n = tri_expand(p, xp, l, wl);
    for (int q = 0; q < n; q++) {
        x[q] = (double)l[q][1];
        y[q] = (double)l[q][2];
        w[q] = (double)wl[q];
    }
    return n;
}

/* ---------------------------------------------------------- basis */
/* Values and reference derivatives of all shape functions at one point.
 * phi: [4][NS]; row 0 values, rows 1..3 d/dxi, d/deta, d/dzeta. */
static void basis_point(int elem, int p, const double *pt, double *phi) {
    if (elem == ORC_TET) {
        double x = pt[0], y = pt[1], z = pt[2];
        double v[4] = {1.0 - x - y - z, x, y, z};
        double d[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 0, 1}};
        for (int i = 0; i < 4; i++) {
            phi[i] = v[i];
            for (int k = 0; k < 3; k++) phi[(1 + k) * 4 + i] = d[k][i];
        }
        return;
    }
    int NS = orc_ns(elem, p), NT = (p + 1) * (p + 2) / 2;
    ld xi = pt[0], eta = pt[1], zeta = pt[2];
    ld r = 2.0L * xi - 1.0L, s = 2.0L * eta - 1.0L;
    ld a = 2.0L * (1.0L + r) / (1.0L - s) - 1.0L, bb = s;
    ld tv[64], tx[64], ty[64];
    int t = 0;
    for (int nn = 0; nn <= p; nn++)
        for (int i = nn; i >= 0; i--, t++) {
            int j = nn - i;
            ld fa = jacobi_l(i, 0, 0, a), dfa = djacobi_l(i, 0, 0, a);
            ld hb = (1.0L - bb) / 2.0L;
            ld pj = jacobi_l(j, 2 * i + 1, 0, bb), dpj = djacobi_l(j, 2 * i + 1, 0, bb);
            ld gb = ipow_l(hb, i) * pj;
            ld dgb = (i > 0 ? -0.5L * (ld)i * ipow_l(hb, i - 1) * pj : 0.0L) + ipow_l(hb, i) * dpj;
            ld dpsi_da = dfa * gb, dpsi_db = fa * dgb;
            ld dpsi_dr = dpsi_da * 2.0L / (1.0L - s);
            ld dpsi_ds = dpsi_da * 2.0L * (1.0L + r) / ((1.0L - s) * (1.0L - s)) + dpsi_db;
            tv[t] = fa * gb;
            tx[t] = 2.0L * dpsi_dr;
            ty[t] = 2.0L * dpsi_ds;
        }
    for (int k = 0; k <= p; k++) {
        ld L = jacobi_l(k, 0, 0, zeta), dL = djacobi_l(k, 0, 0, zeta);
        for (int tt = 0; tt < NT; tt++) {
            int i = tt + NT * k;
            phi[0 * NS + i] = (double)(tv[tt] * L);
            phi[1 * NS + i] = (double)(tx[tt] * L);
            phi[2 * NS + i] = (double)(ty[tt] * L);
            phi[3 * NS + i] = (double)(tv[tt] * dL);
        }
    }
}

/* phi: [npts][4][NS] */
int orc_basis(int elem, int p, int npts, const double *pts, double *phi) {
    int NS = orc_ns(elem, p);
    if (NS < 0) return -1;
    for (int q = 0; q < npts; q++) basis_point(elem, p, pts + 3 * q, phi + (size_t)q * 4 * NS);
    return NS;
}

/* ------------------------------------------------------ geometry map */
/* Vertex shape functions N_v of the reference->real map and their
 * reference derivatives dN[k][v] at one point. */
static int map_derivs(int elem, const double *pt, double dN[3][6]) {
    if (elem == ORC_TET) {
        double d[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 0, 1}};
        for (int k = 0; k < 3; k++)
            for (int v = 0; v < 4; v++) dN[k][v] = d[k][v];
        return 4;
    }
    double xi = pt[0], eta = pt[1], zeta = pt[2];
    double lam[3] = {1.0 - xi - eta, xi, eta};
    double dlx[3] = {-1.0, 1.0, 0.0}, dly[3] = {-1.0, 0.0, 1.0};
    double lo = (1.0 - zeta) / 2.0, hi = (1.0 + zeta) / 2.0;
    for (int a = 0; a < 3; a++) {
        /* N_a = lam_a (1-zeta)/2 ; N_{a+3} = lam_a (1+zeta)/2 */
        dN[0][a] = dlx[a] * lo;
        dN[1][a] = dly[a] * lo;
        dN[2][a] = -0.5 * lam[a];
        dN[0][a + 3] = dlx[a] * hi;
        dN[1][a + 3] = dly[a] * hi;
        dN[2][a + 3] = 0.5 * lam[a];
    }
    return 6;
}

static double det3(const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* inverse by cofactors: Ji[k][m] = cof(J)[m][k] / det */
static void inv3(const double J[3][3], double det, double Ji[3][3]) {
    for (int k = 0; k < 3; k++)
        for (int m = 0; m < 3; m++) {
            int r0 = (m + 1) % 3, r1 = (m + 2) % 3, c0 = (k + 1) % 3, c1 = (k + 2) % 3;
            Ji[k][m] = (J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0]) / det;
        }
}

/* Jacobian terms (Section 4: the NOJAC kernel variants read them instead of
 * computing them): for every element and quadrature point, det J and the 9
 * entries of J^{-1}.  terms[e][q][0] = det J, terms[e][q][1 + 3k + m] =
 * (J^{-1})[k][m] = d xi_k / d x_m.  status[e]: ORC_ST_NONFINITE for a
 * non-finite coordinate, ORC_ST_DET if det J <= 0 (or NaN) at some point. */
int orc_jacobian_terms(int elem, int p, int64_t E, const double *coords, double *terms,
                       int32_t *status) {
    int NQ = orc_nq(elem, p);
    if (NQ < 0) return -1;
    int nv = elem == ORC_TET ? 4 : 6;
    double *xq = (double *)malloc(sizeof(double) * 3 * NQ);
    double *wq = (double *)malloc(sizeof(double) * NQ);
    orc_rule(elem, p, xq, wq);
    for (int64_t e = 0; e < E; e++) {
        const double *X = coords + (size_t)e * nv * 3;
        int32_t st = 0;
        for (int k = 0; k < nv * 3; k++)
            if (!isfinite(X[k])) st |= ORC_ST_NONFINITE;
        for (int q = 0; q < NQ; q++) {
            double dN[3][6], J[3][3], Ji[3][3];
            map_derivs(elem, xq + 3 * q, dN);
            for (int i = 0; i < 3; i++)
                for (int k = 0; k < 3; k++) {
                    double s = 0.0;
                    for (int v = 0; v < nv; v++) s += X[3 * v + i] * dN[k][v];
                    J[i][k] = s;
                }
            double det = det3(J);
            if (!(det > 0.0)) st |= ORC_ST_DET;
            inv3(J, det, Ji);
            double *t = terms + ((size_t)e * NQ + q) * 10;
            t[0] = det;
            for (int k = 0; k < 3; k++)
                for (int m = 0; m < 3; m++) t[1 + 3 * k + m] = Ji[k][m];
        }
        if (status) status[e] = st;
    }
    free(xq);
    free(wq);
    return 0;
}

/* ------------------------------------------------ nonlinear coefficient law */
/* k solves F(k) = k - 1 - 0.5 exp(-u^2) - 0.2 log(1 + k g) = 0; exactly 8
 * Newton steps from k0 = 1 + 0.5 exp(-u^2), no early exit. */
double orc_law_k(double u, double g) {
    double e = 0.5 * exp(-u * u);
    double k = 1.0 + e;
    for (int it = 0; it < 8; it++) {
        double F = k - 1.0 - e - 0.2 * log(1.0 + k * g);
        double Fp = 1.0 - 0.2 * g / (1.0 + k * g);
        k -= F / Fp;
    }
    return k;
}

double orc_law_residual(double u, double g, double k) {
    return k - 1.0 - 0.5 * exp(-u * u) - 0.2 * log(1.0 + k * g);
}

/* -------------------------------------------------- MLP surrogate (FP64) */
/* 2 -> H -> H -> 1 with tanh.  Parameter vector layout (row-major):
 *   W1[H][2], b1[H], W2[H][H], b2[H], W3[1][H], b3[1].
 * Inputs are u and s = |grad u|, normalised to [-1,1]^2 over the box
 * [u0,u1] x [s0,s1]: u linearly, s linearly in log s (the law depends on s
 * through log(1 + k s^2)). */
static void mlp_inputs(const double *box, double u, double s, double *x0, double *x1) {
    *x0 = 2.0 * (u - box[0]) / (box[1] - box[0]) - 1.0;
    *x1 = 2.0 * (log(s) - log(box[2])) / (log(box[3]) - log(box[2])) - 1.0;
}

static double mlp_forward(int H, const double *th, const double *box, double u, double s,
                          double *h1, double *h2) {
    const double *W1 = th, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H,
                 *b3 = W3 + H;
    double x0, x1;
    mlp_inputs(box, u, s, &x0, &x1);
    for (int i = 0; i < H; i++) h1[i] = tanh(W1[2 * i] * x0 + W1[2 * i + 1] * x1 + b1[i]);
    for (int i = 0; i < H; i++) {
        double a = b2[i];
        for (int j = 0; j < H; j++) a += W2[i * H + j] * h1[j];
        h2[i] = tanh(a);
    }
    double y = b3[0];
    for (int j = 0; j < H; j++) y += W3[j] * h2[j];
    return y;
}

int orc_mlp_nparams(int H) { return 2 * H + H + H * H + H + H + 1; }

/* y[i] = MLP(u[i], s[i]) */
void orc_mlp_forward(int H, const double *th, const double *box, int64_t n, const double *u,
                     const double *s, double *y) {
    double h1[256], h2[256];
    for (int64_t i = 0; i < n; i++) y[i] = mlp_forward(H, th, box, u[i], s[i], h1, h2);
}

/* Loss L = mean_s (y_s - t_s)^2 and its gradient dL/dtheta by backpropagation
 * (reverse-mode chain rule through the three layers). */
double orc_mlp_loss_grad(int H, const double *th, const double *box, int64_t n, const double *u,
                         const double *sv, const double *t, double *grad) {
    const double *W2 = th + 3 * H, *W3 = th + 3 * H + H * H + H;
    int P = orc_mlp_nparams(H);
    double *gW1 = grad, *gb1 = gW1 + 2 * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H,
           *gb3 = gW3 + H;
    memset(grad, 0, sizeof(double) * P);
    double h1[256], h2[256], d2[256], d1[256], L = 0.0;
    for (int64_t s = 0; s < n; s++) {
        double y = mlp_forward(H, th, box, u[s], sv[s], h1, h2);
        double x0, x1;
        mlp_inputs(box, u[s], sv[s], &x0, &x1);
        double r = y - t[s];
        L += r * r;
        double dy = 2.0 * r / (double)n;
        gb3[0] += dy;
        for (int j = 0; j < H; j++) {
            gW3[j] += dy * h2[j];
            d2[j] = dy * W3[j] * (1.0 - h2[j] * h2[j]);
        }
        for (int i = 0; i < H; i++) {
            gb2[i] += d2[i];
            for (int j = 0; j < H; j++) gW2[i * H + j] += d2[i] * h1[j];
        }
        for (int j = 0; j < H; j++) {
            double s2 = 0.0;
            for (int i = 0; i < H; i++) s2 += W2[i * H + j] * d2[i];
            d1[j] = s2 * (1.0 - h1[j] * h1[j]);
        }
        for (int i = 0; i < H; i++) {
            gb1[i] += d1[i];
            gW1[2 * i] += d1[i] * x0;
            gW1[2 * i + 1] += d1[i] * x1;
        }
    }
    return L / (double)n;
}

/* ------------------------------------------------ element integration */
/* Geometry at one reference point (Section 2, the reference-to-real map):
 * J[i][k] = d x_i / d xi_k = sum_v x_v[i] dN_v/dxi_k, det J, and Ji = J^{-1}. */
static double point_geometry(int elem, const double *X, const double *xi, double Ji[3][3]) {
    int nv = elem == ORC_TET ? 4 : 6;
    double dN[3][6], J[3][3];
    map_derivs(elem, xi, dN);
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) {
            double s = 0.0;
            for (int v = 0; v < nv; v++) s += X[3 * v + i] * dN[k][v];
            J[i][k] = s;
        }
    double det = det3(J);
    inv3(J, det, Ji);
    return det;
}

/* Physical shape-function table at a point (eq. sum_int, chain rule):
 * psi[0][i] = phi[0][i], psi[1+m][i] = sum_k (J^{-1})[k][m] phi[1+k][i]. */
static void physical_table(int NS, const double *phi, const double Ji[3][3], double *psi) {
    for (int i = 0; i < NS; i++) {
        psi[i] = phi[i];
        for (int m = 0; m < 3; m++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += Ji[k][m] * phi[(1 + k) * NS + i];
            psi[(1 + m) * NS + i] = s;
        }
    }
}

/* Diffusion coefficient that depends on the previous solution (Section 2: the
 * coefficients at a point may be computed from the old degrees of freedom).
 * The field and its physical gradient at the point, from the element's
 * coefficient vector U and the physical table psi:
 *   u = sum_i U_i psi[0][i],  grad u = sum_i U_i psi[1..3][i],  s = |grad u|;
 * law 1: k = law_k(u, s^2) (the exact law in the squared gradient);
 * law 2: k = MLP(u, s) if (u, s) lies in the network's box, else the exact
 * law and ORC_ST_FALLBACK.  Returns the status bits. */
static int32_t point_law(int NS, const double *psi, const double *U, int law, int H,
                         const double *theta, const double *box, double *u_out, double *s_out,
                         double *k_out, double *h1, double *h2) {
    double u = 0.0, gu[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NS; i++) {
        u += U[i] * psi[i];
        for (int m = 0; m < 3; m++) gu[m] += U[i] * psi[(1 + m) * NS + i];
    }
    double g = gu[0] * gu[0] + gu[1] * gu[1] + gu[2] * gu[2];
    double s = sqrt(g), k;
    int32_t st = 0;
    if (law == 2 && u >= box[0] && u <= box[1] && s >= box[2] && s <= box[3]) {
        k = mlp_forward(H, theta, box, u, s, h1, h2);
    } else {
        k = orc_law_k(u, g);
        if (law == 2) st |= ORC_ST_FALLBACK;
    }
    *u_out = u;
    *s_out = s;
    *k_out = k;
    return st;
}

/* Coefficient matrix C[iD][jD] of the generic form at a point (Section 2,
 * -div(D grad u) + b.grad u + c u = f; iD = 0 value, 1..3 derivatives, row =
 * test function): C[0][0] = c, C[0][1+m] = b_m, C[1+l][1+m] = D[l][m]
 * (D = k I when the law gives k), C[1+l][0] = 0. */
static void coefficient_matrix(const double *cf, int law, double k, double C[4][4]) {
    memset(C, 0, sizeof(double) * 16);
    C[0][0] = cf[9];
    for (int m = 0; m < 3; m++) C[0][1 + m] = cf[6 + m];
    if (law == 0) {
        double D[3][3] = {{cf[0], cf[3], cf[4]}, {cf[3], cf[1], cf[5]}, {cf[4], cf[5], cf[2]}};
        for (int l = 0; l < 3; l++)
            for (int m = 0; m < 3; m++) C[1 + l][1 + m] = D[l][m];
    } else {
        for (int l = 0; l < 3; l++) C[1 + l][1 + l] = k;
    }
}

static int32_t nonfinite_inputs(const double *X, int nv, const double *cf, int ncf) {
    int32_t st = 0;
    for (int k = 0; k < nv * 3; k++)
        if (!isfinite(X[k])) st |= ORC_ST_NONFINITE;
    for (int k = 0; k < ncf; k++)
        if (!isfinite(cf[k])) st |= ORC_ST_NONFINITE;
    return st;
}

/* Element matrix and load vector by the quadrature sum of the weak form
 * (eq. sum_int):
 *   A^e[i][j] = sum_Q w_Q det J_Q sum_{iD,jD} psi_Q[iD][i] C_Q[iD][jD] psi_Q[jD][j],
 *   b^e[i]    = sum_Q w_Q det J_Q f psi_Q[0][i]   (the load vector; the paper
 *                                                  integrates only A^e).
 * law: 0 constant coefficients; 1 exact nonlinear law, D = k I; 2 network
 * inside its box [u0,u1] x [s0,s1], exact law outside (status bit 8).
 * coords [E][nv][3]; coeffs SoA [11][cstride]: Dxx Dyy Dzz Dxy Dxz Dyz bx by bz c f;
 * ucoef [E][NS] (law != 0); A [E][NS][NS]; b [E][NS]; status [E] (nullable). */
int orc_integrate_ex(int elem, int p, int64_t E, const double *coords, const double *coeffs,
                     int64_t cstride, int law, const double *ucoef, int H, const double *theta,
                     const double *box, double *A, double *bvec, int32_t *status, int nthreads) {
    int NS = orc_ns(elem, p), NQ = orc_nq(elem, p);
    if (NS < 0 || NQ < 0) return -1;
    int nv = elem == ORC_TET ? 4 : 6;
    double *xq = (double *)malloc(sizeof(double) * 3 * NQ);
    double *wq = (double *)malloc(sizeof(double) * NQ);
    double *phiQ = (double *)malloc(sizeof(double) * (size_t)NQ * 4 * NS);
    orc_rule(elem, p, xq, wq);
    orc_basis(elem, p, NQ, xq, phiQ);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *psi = (double *)malloc(sizeof(double) * 4 * NS);
        double *Cpsi = (double *)malloc(sizeof(double) * 4 * NS);
        double h1[256], h2[256];
#pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < E; e++) {
            const double *X = coords + (size_t)e * nv * 3;
            double cf[11];
            for (int k = 0; k < 11; k++) cf[k] = coeffs[(size_t)k * cstride + e];
            int32_t st = nonfinite_inputs(X, nv, cf, 11);
            double *Ae = A + (size_t)e * NS * NS, *be = bvec + (size_t)e * NS;
            memset(Ae, 0, sizeof(double) * NS * NS);
            memset(be, 0, sizeof(double) * NS);
            for (int q = 0; q < NQ; q++) {
                double Ji[3][3], C[4][4], k = 0.0;
                double det = point_geometry(elem, X, xq + 3 * q, Ji);
                if (!(det > 0.0)) st |= ORC_ST_DET;
                physical_table(NS, phiQ + (size_t)q * 4 * NS, Ji, psi);
                if (law != 0) {
                    double u, s;
                    st |= point_law(NS, psi, ucoef + (size_t)e * NS, law, H, theta, box, &u, &s,
                                    &k, h1, h2);
                }
                coefficient_matrix(cf, law, k, C);
                double dw = wq[q] * det;
                /* (C psi)[iD][j] = sum_jD C[iD][jD] psi[jD][j] */
                for (int iD = 0; iD < 4; iD++)
                    for (int j = 0; j < NS; j++) {
                        double s = 0.0;
                        for (int jD = 0; jD < 4; jD++) s += C[iD][jD] * psi[jD * NS + j];
                        Cpsi[iD * NS + j] = s;
                    }
                for (int i = 0; i < NS; i++)
                    for (int j = 0; j < NS; j++) {
                        double s = 0.0;
                        for (int iD = 0; iD < 4; iD++) s += psi[iD * NS + i] * Cpsi[iD * NS + j];
                        Ae[i * NS + j] += dw * s;
                    }
                for (int i = 0; i < NS; i++) be[i] += dw * cf[10] * psi[i];
            }
            if (status) status[e] = st;
        }
        free(psi);
        free(Cpsi);
    }
    free(xq);
    free(wq);
    free(phiQ);
    return 0;
}

/* The law's quantities at every quadrature point (the per-point stage of
 * orc_integrate_ex with law 1 or 2): u [E][NQ], s = |grad u| [E][NQ] and the
 * coefficient k [E][NQ]; status [E] (nullable) as in orc_integrate_ex. */
int orc_point_law(int elem, int p, int64_t E, const double *coords, const double *ucoef, int law,
                  int H, const double *theta, const double *box, double *u_out, double *s_out,
                  double *k_out, int32_t *status) {
    int NS = orc_ns(elem, p), NQ = orc_nq(elem, p);
    if (NS < 0 || NQ < 0 || (law != 1 && law != 2)) return -1;
    int nv = elem == ORC_TET ? 4 : 6;
    double *xq = (double *)malloc(sizeof(double) * 3 * NQ);
    double *wq = (double *)malloc(sizeof(double) * NQ);
    double *phiQ = (double *)malloc(sizeof(double) * (size_t)NQ * 4 * NS);
    double *psi = (double *)malloc(sizeof(double) * 4 * NS);
    double h1[256], h2[256];
    orc_rule(elem, p, xq, wq);
    orc_basis(elem, p, NQ, xq, phiQ);
    for (int64_t e = 0; e < E; e++) {
        const double *X = coords + (size_t)e * nv * 3;
        int32_t st = nonfinite_inputs(X, nv, NULL, 0);
        for (int q = 0; q < NQ; q++) {
            double Ji[3][3];
            double det = point_geometry(elem, X, xq + 3 * q, Ji);
            if (!(det > 0.0)) st |= ORC_ST_DET;
            physical_table(NS, phiQ + (size_t)q * 4 * NS, Ji, psi);
            size_t o = (size_t)e * NQ + q;
            st |= point_law(NS, psi, ucoef + (size_t)e * NS, law, H, theta, box, u_out + o,
                            s_out + o, k_out + o, h1, h2);
        }
        if (status) status[e] = st;
    }
    free(psi);
    free(xq);
    free(wq);
    free(phiQ);
    return 0;
}

/* ------------------------------------------ linear elastostatics (Section 5.1) */
/* Isotropic elasticity, N_E = 3 (Section 5.1, with eq. sum_int per pair of
 * components): block (iE, jE) of A^e couples test component iE with trial
 * component jE,
 *   A[iE][jE][s][r] = sum_Q w_Q det J_Q sum_{l,m} psi_Q[1+l][s] c_{iE l jE m} psi_Q[1+m][r],
 *   c_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk),
 * lam = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu)), constant per
 * element (the paper's material data: Young modulus and Poisson ratio); body
 * force load b[iE][s] = sum_Q w_Q det J_Q f_iE psi_Q[0][s].
 * coeffs SoA [5][cstride]: E, nu, fx, fy, fz.  A [E][3][3][NS][NS], b [E][3][NS].
 * elem: ORC_PRISM (collapsed rule) or ORC_PRISM_T1 (the paper's rule). */
int orc_integrate_elastic_ex(int elem, int p, int64_t E, const double *coords, const double *coeffs,
                             int64_t cstride, double *A, double *bvec, int32_t *status, int nthreads) {
    if (elem != ORC_PRISM && elem != ORC_PRISM_T1) return -1;
    int NS = orc_ns(elem, p), NQ = orc_nq(elem, p);
    if (NS < 0 || NQ < 0) return -1;
    double *xq = (double *)malloc(sizeof(double) * 3 * NQ);
    double *wq = (double *)malloc(sizeof(double) * NQ);
    double *phiQ = (double *)malloc(sizeof(double) * (size_t)NQ * 4 * NS);
    orc_rule(elem, p, xq, wq);
    orc_basis(elem, p, NQ, xq, phiQ);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *psi = (double *)malloc(sizeof(double) * 4 * NS);
#pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < E; e++) {
            const double *X = coords + (size_t)e * 18;
            double cf[5];
            for (int k = 0; k < 5; k++) cf[k] = coeffs[(size_t)k * cstride + e];
            double Ey = cf[0], nu = cf[1];
            double lam = Ey * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = Ey / (2.0 * (1.0 + nu));
            int32_t st = nonfinite_inputs(X, 6, cf, 5);
            /* c[iE][jE][l][m] = c_{iE l jE m} */
            double c[3][3][3][3];
            for (int i = 0; i < 3; i++)
                for (int k = 0; k < 3; k++)
                    for (int j = 0; j < 3; j++)
                        for (int l = 0; l < 3; l++)
                            c[i][k][j][l] = lam * (i == j) * (k == l) +
                                            mu * ((i == k) * (j == l) + (i == l) * (j == k));
            double *Ae = A + (size_t)e * 9 * NS * NS, *be = bvec + (size_t)e * 3 * NS;
            memset(Ae, 0, sizeof(double) * 9 * NS * NS);
            memset(be, 0, sizeof(double) * 3 * NS);
            for (int q = 0; q < NQ; q++) {
                double Ji[3][3];
                double det = point_geometry(elem, X, xq + 3 * q, Ji);
                if (!(det > 0.0)) st |= ORC_ST_DET;
                physical_table(NS, phiQ + (size_t)q * 4 * NS, Ji, psi);
                double dw = wq[q] * det;
                for (int iE = 0; iE < 3; iE++)
                    for (int jE = 0; jE < 3; jE++) {
                        double *blk = Ae + ((size_t)iE * 3 + jE) * NS * NS;
                        for (int s2 = 0; s2 < NS; s2++)
                            for (int r = 0; r < NS; r++) {
                                double sacc = 0.0;
                                for (int l = 0; l < 3; l++)
                                    for (int m = 0; m < 3; m++)
                                        sacc += psi[(1 + l) * NS + s2] * c[iE][jE][l][m] *
                                                psi[(1 + m) * NS + r];
                                blk[s2 * NS + r] += dw * sacc;
                            }
                    }
                for (int iE = 0; iE < 3; iE++)
                    for (int s2 = 0; s2 < NS; s2++) be[iE * NS + s2] += dw * cf[2 + iE] * psi[s2];
            }
            if (status) status[e] = st;
        }
        free(psi);
    }
    free(xq);
    free(wq);
    free(phiQ);
    return 0;
}

/* elasticity on prisms with the collapsed rule */
int orc_integrate_elastic(int p, int64_t E, const double *coords, const double *coeffs,
                          int64_t cstride, double *A, double *bvec, int32_t *status, int nthreads) {
    return orc_integrate_elastic_ex(ORC_PRISM, p, E, coords, coeffs, cstride, A, bvec, status, nthreads);
}

int orc_integrate(int elem, int p, int64_t E, const double *coords, const double *coeffs,
                  int64_t cstride, double *A, double *bvec, int32_t *status, int nthreads) {
    return orc_integrate_ex(elem, p, E, coords, coeffs, cstride, 0, NULL, 0, NULL, NULL, A, bvec,
                            status, nthreads);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
