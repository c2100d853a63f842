// Host construction of quadrature rules and shape-function tables (FP64).
//
// Section 2: quadrature points xi^Q and weights w^Q on the reference element,
// and phi^Q[iQ][iD][iDOF], the shape functions (iD = 0) and their derivatives
// with respect to reference coordinates (iD = 1..3) at every point.  These are
// the same for all elements of one degree, so they are computed once and kept
// in device memory (Section 4.1).
//
// Gauss rules: Golub-Welsch (nodes = eigenvalues of the symmetric Jacobi
// matrix of the orthogonal-polynomial recurrence, weights = mu_0 times the
// squared first components of the normalised eigenvectors), with the small
// dense eigenproblem solved by cyclic Jacobi rotations; each node is then
// polished by Newton steps on the three-term recurrence and its weight
// recomputed from the Christoffel function (a sum of positive terms, more
// accurate than the eigenvector component).
//
// Basis: Dubiner triangle functions in collapsed coordinates times Legendre
// polynomials in zeta; Jacobi polynomials and their derivatives are evaluated
// by the three-term recurrence differentiated in forward mode.  The collapsed
// chain rule is written so that no division by (1 - b) occurs:
//   psi = P_i(a) h^i Q_j(b),  h = (1-b)/2,  Q_j = P_j^(2i+1,0)
//   d psi/d xi  = 2 P_i'(a) h^(i-1) Q_j(b)
//   d psi/d eta = h^(i-1) [(1+a) P_i'(a) - i P_i(a)] Q_j(b) + 2 h^i P_i(a) Q_j'(b)
#include <cmath>
#include <cstring>
#include <vector>

#include "fem_internal.h"

namespace fem {
namespace {

// P_n^(a,b)(x) and its derivative by the three-term recurrence.
void jacobi_rec(int n, double al, double be, double x, double *P, double *dP) {
  double p0 = 1.0, d0 = 0.0;
  if (n == 0) {
    *P = p0;
    *dP = d0;
    return;
  }
  double p1 = 0.5 * ((al + be + 2.0) * x + (al - be)), d1 = 0.5 * (al + be + 2.0);
  for (int k = 2; k <= n; k++) {
    double s = 2.0 * k + al + be;
    double c1 = 2.0 * k * (k + al + be) * (s - 2.0);
    double c2 = (s - 1.0) * (al * al - be * be);
    double c3 = (s - 2.0) * (s - 1.0) * s;
    double c4 = 2.0 * (k + al - 1.0) * (k + be - 1.0) * s;
    double p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
    double d2 = ((c2 + c3 * x) * d1 + c3 * p1 - c4 * d0) / c1;
    p0 = p1;
    d0 = d1;
    p1 = p2;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

// Golub-Welsch Gauss-Jacobi rule with n points for weight (1-x)^al (1+x)^be.
void gauss_jacobi_gw(int n, double al, double be, double *x, double *w) {
  double A[16][16], V[16][16];
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      A[i][j] = 0.0;
      V[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int k = 0; k < n; k++) {
    double s = 2.0 * k + al + be;
    A[k][k] = (k == 0) ? (be - al) / (al + be + 2.0) : (be * be - al * al) / (s * (s + 2.0));
    if (k >= 1) {
      double num = 4.0 * k * (k + al) * (k + be) * (k + al + be);
      double den = s * s * (s + 1.0) * (s - 1.0);
      A[k][k - 1] = A[k - 1][k] = std::sqrt(num / den);
    }
  }
  // cyclic Jacobi rotations until the off-diagonal part vanishes
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) off += A[i][j] * A[i][j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; k++) {  // A <- A R (columns p, q)
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {  // A <- R^T A (rows p, q)
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  double mu0 = std::pow(2.0, al + be + 1.0) * std::tgamma(al + 1.0) * std::tgamma(be + 1.0) /
               std::tgamma(al + be + 2.0);
  // sort ascending
  int idx[16];
  for (int i = 0; i < n; i++) idx[i] = i;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) std::swap(idx[i], idx[j]);
  for (int i = 0; i < n; i++) {
    int k = idx[i];
    double z = A[k][k];
    for (int it = 0; it < 3; it++) {  // polish the node
      double P, dP;
      jacobi_rec(n, al, be, z, &P, &dP);
      if (dP != 0.0) z -= P / dP;
    }
    x[i] = z;
    // weight from the Christoffel function at the polished node,
    // 1/w = sum_{m<n} P_m(z)^2 / h_m, h_m = int (1-x)^al (1+x)^be P_m^2;
    // the eigenvector weight is the fallback if the sum is not usable
    double inv = 0.0;
    for (int m = 0; m < n; m++) {
      double P, dP;
      jacobi_rec(m, al, be, z, &P, &dP);
      const double hm = std::pow(2.0, al + be + 1.0) / (2.0 * m + al + be + 1.0) *
                        std::tgamma(m + al + 1.0) * std::tgamma(m + be + 1.0) /
                        (std::tgamma(m + al + be + 1.0) * std::tgamma(m + 1.0));
      inv += P * P / hm;
    }
    w[i] = (inv > 0.0 && std::isfinite(inv)) ? 1.0 / inv : mu0 * V[0][k] * V[0][k];
  }
}

void prism_basis_point(int p, double xi, double eta, double zeta, double *phi, int ns) {
  const int nt = (p + 1) * (p + 2) / 2;
  const double r = 2.0 * xi - 1.0, s = 2.0 * eta - 1.0;
  const double h = 0.5 * (1.0 - s);      // (1-b)/2 with b = s
  const double a = (1.0 + r) / h - 1.0;  // 2(1+r)/(1-s) - 1
  double tv[64], tx[64], ty[64];
  int t = 0;
  for (int n = 0; n <= p; n++)
    for (int i = n; i >= 0; i--, t++) {
      int j = n - i;
      double Pi, dPi, Qj, dQj;
      jacobi_rec(i, 0.0, 0.0, a, &Pi, &dPi);
      jacobi_rec(j, 2.0 * i + 1.0, 0.0, s, &Qj, &dQj);
      double hi1 = 1.0;  // h^(i-1) for i >= 1
      for (int k = 1; k < i; k++) hi1 *= h;
      double hi = (i >= 1) ? hi1 * h : 1.0;
      tv[t] = Pi * hi * Qj;
      if (i == 0) {
        tx[t] = 0.0;
        ty[t] = 2.0 * dQj;  // d/deta of Q_j(2 eta - 1)
      } else {
        tx[t] = 2.0 * dPi * hi1 * Qj;
        ty[t] = hi1 * ((1.0 + a) * dPi - i * Pi) * Qj + 2.0 * hi * Pi * dQj;
      }
    }
  for (int k = 0; k <= p; k++) {
    double L, dL;
    jacobi_rec(k, 0.0, 0.0, zeta, &L, &dL);
    for (int tt = 0; tt < nt; tt++) {
      int dof = tt + nt * k;
      phi[0 * ns + dof] = tv[tt] * L;
      phi[1 * ns + dof] = tx[tt] * L;
      phi[2 * ns + dof] = ty[tt] * L;
      phi[3 * ns + dof] = tv[tt] * dL;
    }
  }
}

// Fully symmetric positive-interior triangle rules of degree 2p behind the
// paper's prism rules (Table 1), as orbit parameters in barycentric
// coordinates; written by tri_rules_gen.cpp (which documents how they are
// found and chosen).
struct TriRuleRow {
  int p, n0, n1, n2;
  double v[24];
};
const TriRuleRow kTriRules[] = {
#include "fem_tri_rules.inc"
};

// Points (xi, eta) = (l1, l2) and weights of the degree-2p symmetric
// triangle rule: the centroid, then each S21 orbit (a, a, c), (a, c, a),
// (c, a, a), then each S111 orbit in the six permutations of (a, b, c).
// Checks exactness on every monomial xi^i eta^j, i + j <= 2p, against
// i! j! / (i + j + 2)!; false if a table row is missing or inexact.
bool tri_rule_table1(int p, std::vector<double> &x, std::vector<double> &y, std::vector<double> &w) {
  const TriRuleRow *r = nullptr;
  for (const TriRuleRow &row : kTriRules)
    if (row.p == p) r = &row;
  if (!r) return false;
  x.clear();
  y.clear();
  w.clear();
  auto add = [&](double l1, double l2, double wt) {
    x.push_back(l1);
    y.push_back(l2);
    w.push_back(wt);
  };
  int k = 0;
  for (int o = 0; o < r->n0; o++, k++) add(1.0 / 3.0, 1.0 / 3.0, r->v[k]);
  for (int o = 0; o < r->n1; o++, k += 2) {
    const double a = r->v[k], c = 1.0 - 2.0 * a, wt = r->v[k + 1];
    add(a, c, wt);  // (l0, l1, l2) = (a, a, c)
    add(c, a, wt);  // (a, c, a)
    add(a, a, wt);  // (c, a, a)
  }
  for (int o = 0; o < r->n2; o++, k += 3) {
    const double a = r->v[k], b = r->v[k + 1], c = 1.0 - a - b, wt = r->v[k + 2];
    const double l[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
    for (int m = 0; m < 6; m++) add(l[m][1], l[m][2], wt);
  }
  if ((int)w.size() != ntri_of(p, FEM_RULE_TABLE1)) return false;
  for (int i = 0; i <= 2 * p; i++)
    for (int j = 0; i + j <= 2 * p; j++) {
      long double sum = 0.0L, ex = 1.0L;
      for (int m = 2; m <= i; m++) ex *= m;
      for (int m = 2; m <= j; m++) ex *= m;
      for (int m = 2; m <= i + j + 2; m++) ex /= m;
      for (size_t q = 0; q < w.size(); q++)
        sum += (long double)w[q] * std::pow((long double)x[q], i) * std::pow((long double)y[q], j);
      if (std::fabs((double)(sum / ex - 1.0L)) > 1e-13) return false;
    }
  return true;
}

}  // namespace

bool build_host_rule(int elem, int p, HostRule *out, int rule) {
  if (elem == FEM_TET4) {
    if (p != 1 || rule != FEM_RULE_COLLAPSED) return false;
    out->nq = 4;
    out->ns = 4;
    // 4-point degree-2 rule: barycentric (al, be, be, be) and permutations
    const double al = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, be = (5.0 - std::sqrt(5.0)) / 20.0;
    const double pts[4][3] = {{be, be, be}, {al, be, be}, {be, al, be}, {be, be, al}};
    out->xi.assign(&pts[0][0], &pts[0][0] + 12);
    out->w.assign(4, 1.0 / 24.0);
    out->phi.assign(4 * 4 * 4, 0.0);
    for (int q = 0; q < 4; q++) {
      double *f = &out->phi[q * 16];
      const double x = pts[q][0], y = pts[q][1], z = pts[q][2];
      const double val[4] = {1.0 - x - y - z, x, y, z};
      const double grad[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      for (int i = 0; i < 4; i++) {
        f[i] = val[i];
        for (int d = 0; d < 3; d++) f[(1 + d) * 4 + i] = grad[i][d];
      }
    }
    return true;
  }
  if (elem != FEM_PRISM6 || p < 1 || p > kMaxP) return false;
  if (rule != FEM_RULE_COLLAPSED && rule != FEM_RULE_TABLE1) return false;
  const int n = p + 1, nq = nq_of(elem, p, rule), ns = ns_of(elem, p);
  double xa[16], wa[16], xb[16], wb[16];
  gauss_jacobi_gw(n, 0.0, 0.0, xa, wa);
  gauss_jacobi_gw(n, 1.0, 0.0, xb, wb);
  out->nq = nq;
  out->ns = ns;
  out->xi.resize(3 * nq);
  out->w.resize(nq);
  out->phi.resize((size_t)nq * 4 * ns);
  if (rule == FEM_RULE_TABLE1) {
    // the paper's prism rule: symmetric triangle rule x Gauss-Legendre in zeta
    std::vector<double> tx, ty, tw;
    if (!tri_rule_table1(p, tx, ty, tw)) return false;
    const int nt = (int)tw.size();
    for (int iz = 0; iz < n; iz++)
      for (int it = 0; it < nt; it++) {
        const int q = iz * nt + it;
        out->xi[3 * q + 0] = tx[it];
        out->xi[3 * q + 1] = ty[it];
        out->xi[3 * q + 2] = xa[iz];
        out->w[q] = tw[it] * wa[iz];
        prism_basis_point(p, tx[it], ty[it], xa[iz], &out->phi[(size_t)q * 4 * ns], ns);
      }
    return true;
  }
  int q = 0;
  for (int iz = 0; iz < n; iz++)
    for (int ia = 0; ia < n; ia++)
      for (int ib = 0; ib < n; ib++, q++) {
        const double xi = 0.25 * (1.0 + xa[ia]) * (1.0 - xb[ib]);
        const double eta = 0.5 * (1.0 + xb[ib]);
        out->xi[3 * q + 0] = xi;
        out->xi[3 * q + 1] = eta;
        out->xi[3 * q + 2] = xa[iz];
        out->w[q] = 0.125 * wa[ia] * wb[ib] * wa[iz];
        prism_basis_point(p, xi, eta, xa[iz], &out->phi[(size_t)q * 4 * ns], ns);
      }
  return true;
}

// Factors of the prism tables for sum factorisation.  The basis function
// t = (i, j) x k is psi_ij(a, b) L_k(zeta) with psi_ij = P_i(a) h^i Q_j(b),
// h = (1 - b)/2, Q_j = P_j^(2i+1,0), and the rule's point (iz, ia, ib) sits at
// a = xa[ia], b = xb[ib], zeta = xa[iz], so every entry of the full table is a
// product of 1D factors (the chain rule of the collapsed coordinates as in
// prism_basis_point):
//   value     Pa[ia][i]  Bq[t][ib] L[iz][k],   Pa = P_i(a),   Bq = h^i Q_j(b)
//   d/dxi     Px[ia][i]  Bx[t][ib] L[iz][k],   Px = 2 P_i'(a), Bx = h^(i-1) Q_j(b)
//   d/deta   (Pe[ia][i]  Bx[t][ib] + Pa[ia][i] By[t][ib]) L[iz][k],
//            Pe = (1 + a) P_i'(a) - i P_i(a),  By = 2 h^i Q_j'(b)
//   d/dzeta   Pa[ia][i]  Bq[t][ib] dL[iz][k]
// (Bx = 0 for i = 0, where Px and Pe vanish).
void build_sf_tables(int p, std::vector<double> &out) {
  const int n = p + 1, nt = n * (n + 1) / 2, np_ = n | 1;
  double xa[16], wa[16], xb[16], wb[16];
  gauss_jacobi_gw(n, 0.0, 0.0, xa, wa);
  gauss_jacobi_gw(n, 1.0, 0.0, xb, wb);
  out.assign((size_t)5 * n * n + (size_t)3 * nt * np_, 0.0);
  double *Pa = out.data(), *Px = Pa + n * n, *Pe = Px + n * n;
  double *Bq = Pe + n * n, *Bx = Bq + nt * np_, *By = Bx + nt * np_;
  double *L = By + nt * np_, *dL = L + n * n;
  for (int ia = 0; ia < n; ia++)
    for (int i = 0; i < n; i++) {
      double P, dP;
      jacobi_rec(i, 0.0, 0.0, xa[ia], &P, &dP);
      Pa[ia * n + i] = P;
      Px[ia * n + i] = 2.0 * dP;
      Pe[ia * n + i] = (1.0 + xa[ia]) * dP - i * P;
    }
  int t = 0;
  for (int m = 0; m <= p; m++)
    for (int i = m; i >= 0; i--, t++) {
      const int j = m - i;
      for (int ib = 0; ib < n; ib++) {
        const double b = xb[ib], h = 0.5 * (1.0 - b);
        double Q, dQ;
        jacobi_rec(j, 2.0 * i + 1.0, 0.0, b, &Q, &dQ);
        double hi1 = 1.0;  // h^(i-1) for i >= 1
        for (int k = 1; k < i; k++) hi1 *= h;
        const double hi = i >= 1 ? hi1 * h : 1.0;
        Bq[t * np_ + ib] = hi * Q;
        Bx[t * np_ + ib] = i >= 1 ? hi1 * Q : 0.0;
        By[t * np_ + ib] = 2.0 * hi * dQ;
      }
    }
  for (int iz = 0; iz < n; iz++)
    for (int k = 0; k < n; k++) {
      double P, dP;
      jacobi_rec(k, 0.0, 0.0, xa[iz], &P, &dP);
      L[iz * n + k] = P;
      dL[iz * n + k] = dP;
    }
}

}  // namespace fem
