// Generator of the fully symmetric triangle rules behind the paper's prism
// rules (Section 2, Table 1: N_Q = 6, 18, 48, 80, 150, 231, 336 points for
// p = 1..7 = (3, 6, 12, 16, 25, 33, 42) triangle points x (p + 1) Gauss-Legendre
// points in zeta).  Writes csrc/fem_tri_rules.inc, which fem_tables.cpp
// includes; the library does not run this program.
//
//   g++ -O2 -fopenmp -std=c++17 tri_rules_gen.cpp -o /tmp/tri_rules_gen &&
//   /tmp/tri_rules_gen > csrc/fem_tri_rules.inc
//
// A fully symmetric rule is made of orbits under the six permutations of the
// barycentric coordinates: the centroid (weight w), S21 orbits (a, a, 1-2a)
// (3 points; a, w) and S111 orbits (a, b, 1-a-b) (6 points; a, b, w).  Degree
// d = 2p exactness for polynomials invariant under the permutations is
// exactness for all polynomials of degree <= d, and the invariant polynomials
// of degree <= d are spanned by e2^i e3^j (2i + 3j <= d; e2, e3 the elementary
// symmetric functions of the barycentric coordinates).  With N points the
// number of orbits of each kind (n0, n1, n2) follows from requiring as many
// unknowns (n0 + 2 n1 + 3 n2) as moment equations: (0,1,0), (0,2,0), (0,2,1),
// (1,3,1), (1,2,3), (0,5,3), (0,6,4) for d = 2..14, the orbit structure of the
// published degree-2p rules with these point counts (Dunavant, Int. J. Numer.
// Meth. Engng 21 (1985) 1129-1148).
//
// The equations are solved here, not copied: homotopy continuation from
// random starts (the target moments move linearly from the start's own
// moments to the exact ones, Newton corrector), in parameters that keep every
// point strictly inside the triangle and every weight positive (a = sigmoid/2
// for S21, softmax for S111, w = exp).  Each path that reaches the exact
// moments gives a positive-interior (PI) rule; the distinct ones are
// collected, polished in long double, and the one whose points keep the
// largest distance from the edges (largest smallest barycentric coordinate)
// is written.  The searches find 1, 1, 2, 1, 4, 2 and 1 distinct PI rules for
// d = 2..14.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

typedef long double LD;

struct Shape {
  int n0, n1, n2;
};
const Shape kShape[8] = {{0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 2, 1}, {1, 3, 1}, {1, 2, 3}, {0, 5, 3}, {0, 6, 4}};
const long kTrials[8] = {0, 20000, 40000, 100000, 200000, 400000, 800000, 3000000};

LD fact(int n) {
  LD r = 1;
  for (int i = 2; i <= n; i++) r *= i;
  return r;
}
// integral of l0^i l1^j l2^k over the reference triangle (area 1/2)
LD dirichlet(int i, int j, int k) { return fact(i) * fact(j) * fact(k) / fact(i + j + k + 2); }
// integral of e2^a e3^b, e2 = l0 l1 + l1 l2 + l2 l0, e3 = l0 l1 l2 (multinomial expansion of e2^a),
// in long double: the final Newton steps solve against these targets
LD moment(int a, int b) {
  LD s = 0;
  for (int x = 0; x <= a; x++)
    for (int y = 0; x + y <= a; y++) {
      const int z = a - x - y;
      s += fact(a) / (fact(x) * fact(y) * fact(z)) * dirichlet(x + z + b, x + y + b, y + z + b);
    }
  return s;
}

struct System {
  Shape sh;
  int nu = 0, ne = 0;
  int ea[64], eb[64];
  LD m[64];
  explicit System(int d) : sh(kShape[d / 2]) {
    nu = sh.n0 + 2 * sh.n1 + 3 * sh.n2;
    for (int b = 0; 3 * b <= d; b++)
      for (int a = 0; 2 * a + 3 * b <= d; a++) {
        ea[ne] = a;
        eb[ne] = b;
        m[ne] = moment(a, b);
        ne++;
      }
  }
};

template <class T>
T ipow(T x, int k) {
  T r = 1;
  for (int i = 0; i < k; i++) r *= x;
  return r;
}

// accumulates an orbit of n points with invariants (e2, e3), derivatives
// de2[], de3[] w.r.t. the orbit's np position unknowns (columns c0..), weight
// wt (dw = d wt / d its unknown, column cw); F[e] and J[e][.] scaled by 1/m[e]
template <class T>
void orbit(const System &S, int n, T e2, T e3, const T *de2, const T *de3, int np, int c0, T wt, T dw, int cw,
           T *F, T (*J)[40]) {
  for (int e = 0; e < S.ne; e++) {
    const int a = S.ea[e], b = S.eb[e];
    const T v = ipow(e2, a) * ipow(e3, b);
    const T g2 = a ? a * ipow(e2, a - 1) * ipow(e3, b) : T(0);
    const T g3 = b ? b * ipow(e3, b - 1) * ipow(e2, a) : T(0);
    const T sc = T(n) / T(S.m[e]);
    F[e] += sc * wt * v;
    J[e][cw] += sc * dw * v;
    for (int q = 0; q < np; q++) J[e][c0 + q] += sc * wt * (g2 * de2[q] + g3 * de3[q]);
  }
}

// moments / exact moments of the rule in unconstrained parameters t
void eval_free(const System &S, const double *t, double *F, double (*J)[40]) {
  for (int e = 0; e < S.ne; e++) {
    F[e] = 0;
    for (int k = 0; k < S.nu; k++) J[e][k] = 0;
  }
  int k = 0;
  for (int o = 0; o < S.sh.n0; o++, k++) {
    const double w = std::exp(t[k]);
    orbit<double>(S, 1, 1.0 / 3, 1.0 / 27, nullptr, nullptr, 0, k, w, w, k, F, J);
  }
  for (int o = 0; o < S.sh.n1; o++, k += 2) {
    const double s = 1 / (1 + std::exp(-t[k])), a = 0.5 * s, da = 0.5 * s * (1 - s), c = 1 - 2 * a;
    const double w = std::exp(t[k + 1]);
    const double de2 = (2 * c - 2 * a) * da, de3 = (2 * a * c - 2 * a * a) * da;
    orbit<double>(S, 3, a * a + 2 * a * c, a * a * c, &de2, &de3, 1, k, w, w, k + 1, F, J);
  }
  for (int o = 0; o < S.sh.n2; o++, k += 3) {
    const double m = std::max(std::max(t[k], t[k + 1]), 0.0);
    const double x1 = std::exp(t[k] - m), x2 = std::exp(t[k + 1] - m), x3 = std::exp(-m), Z = x1 + x2 + x3;
    const double a = x1 / Z, b = x2 / Z, c = x3 / Z, w = std::exp(t[k + 2]);
    const double d2a = b + c, d2b = a + c, d2c = a + b, d3a = b * c, d3b = a * c, d3c = a * b;
    // da/dt1 = a(1-a), db/dt1 = -ab, dc/dt1 = -ac; da/dt2 = -ab, db/dt2 = b(1-b), dc/dt2 = -bc
    const double de2[2] = {d2a * a * (1 - a) - d2b * a * b - d2c * a * c, -d2a * a * b + d2b * b * (1 - b) - d2c * b * c};
    const double de3[2] = {d3a * a * (1 - a) - d3b * a * b - d3c * a * c, -d3a * a * b + d3b * b * (1 - b) - d3c * b * c};
    orbit<double>(S, 6, a * b + b * c + c * a, a * b * c, de2, de3, 2, k, w, w, k + 2, F, J);
  }
}

// the same in the natural parameters (a; a, b; w), long double
void eval_nat(const System &S, const LD *x, LD *F, LD (*J)[40]) {
  for (int e = 0; e < S.ne; e++) {
    F[e] = 0;
    for (int k = 0; k < S.nu; k++) J[e][k] = 0;
  }
  int k = 0;
  for (int o = 0; o < S.sh.n0; o++, k++)
    orbit<LD>(S, 1, LD(1) / 3, LD(1) / 27, nullptr, nullptr, 0, k, x[k], 1, k, F, J);
  for (int o = 0; o < S.sh.n1; o++, k += 2) {
    const LD a = x[k], c = 1 - 2 * a;
    const LD de2 = 2 * c - 2 * a, de3 = 2 * a * c - 2 * a * a;
    orbit<LD>(S, 3, a * a + 2 * a * c, a * a * c, &de2, &de3, 1, k, x[k + 1], 1, k + 1, F, J);
  }
  for (int o = 0; o < S.sh.n2; o++, k += 3) {
    const LD a = x[k], b = x[k + 1], c = 1 - a - b;
    const LD de2[2] = {c - a, c - b}, de3[2] = {b * c - a * b, a * c - a * b};
    orbit<LD>(S, 6, a * b + b * c + c * a, a * b * c, de2, de3, 2, k, x[k + 2], 1, k + 2, F, J);
  }
}

template <class T>
bool solve(int n, T (*A)[40], const T *b, T *x) {
  T M[40][41];
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++) M[i][j] = A[i][j];
    M[i][n] = b[i];
  }
  for (int c = 0; c < n; c++) {
    int pv = c;
    for (int r = c + 1; r < n; r++)
      if (std::fabs(M[r][c]) > std::fabs(M[pv][c])) pv = r;
    if (std::fabs(M[pv][c]) < T(1e-300)) return false;
    if (pv != c)
      for (int q = 0; q <= n; q++) std::swap(M[c][q], M[pv][q]);
    for (int r = c + 1; r < n; r++) {
      const T f = M[r][c] / M[c][c];
      for (int q = c; q <= n; q++) M[r][q] -= f * M[c][q];
    }
  }
  for (int r = n - 1; r >= 0; r--) {
    T s = M[r][n];
    for (int q = r + 1; q < n; q++) s -= M[r][q] * x[q];
    x[r] = s / M[r][r];
  }
  return true;
}

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uni(uint64_t &s) { return (splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }
double gauss(uint64_t &s) { return std::sqrt(-2 * std::log(uni(s) + 1e-300)) * std::cos(6.283185307179586 * uni(s)); }

// one continuation path; false if it fails; natural parameters in x on success
bool path(const System &S, uint64_t seed, LD *x) {
  const int npt = S.sh.n0 + 3 * S.sh.n1 + 6 * S.sh.n2;
  double t[40], F0[64], F[64], J[64][40];
  int k = 0;
  for (int o = 0; o < S.sh.n0; o++) t[k++] = std::log(0.5 / npt) + 0.3 * gauss(seed);
  for (int o = 0; o < S.sh.n1; o++) {
    t[k++] = 1.5 * gauss(seed);
    t[k++] = std::log(0.5 / npt) + 0.3 * gauss(seed);
  }
  for (int o = 0; o < S.sh.n2; o++) {
    t[k++] = 1.2 * gauss(seed);
    t[k++] = 1.2 * gauss(seed);
    t[k++] = std::log(0.5 / npt) + 0.3 * gauss(seed);
  }
  eval_free(S, t, F0, J);
  double tau = 0, dt = 0.01;
  while (tau < 1) {
    const double tn = std::min(1.0, tau + dt);
    double t2[40];
    std::memcpy(t2, t, sizeof(t));
    bool good = false;
    for (int it = 0; it < 6; it++) {
      eval_free(S, t2, F, J);
      double r[64], nr = 0;
      for (int e = 0; e < S.ne; e++) {
        r[e] = (1 - tn) * F0[e] + tn - F[e];
        nr = std::max(nr, std::fabs(r[e]));
      }
      if (!(nr == nr)) break;
      if (nr < 1e-11) {
        good = true;
        break;
      }
      double dx[40], mx = 0;
      if (!solve<double>(S.nu, J, r, dx)) break;
      for (int j = 0; j < S.nu; j++) mx = std::max(mx, std::fabs(dx[j]));
      if (mx > 2) break;
      for (int j = 0; j < S.nu; j++) t2[j] += dx[j];
    }
    double mxp = 0;
    for (int j = 0; j < S.nu; j++) mxp = std::max(mxp, std::fabs(t2[j]));
    if (good && mxp < 40) {
      std::memcpy(t, t2, sizeof(t));
      tau = tn;
      dt = std::min(dt * 1.3, 0.05);
    } else {
      dt *= 0.5;
      if (dt < 1e-6) return false;
    }
  }
  // natural parameters, then Newton in long double on the exact moments
  k = 0;
  for (int o = 0; o < S.sh.n0; o++, k++) x[k] = std::exp((LD)t[k]);
  for (int o = 0; o < S.sh.n1; o++, k += 2) {
    x[k] = 0.5L / (1 + std::exp(-(LD)t[k]));
    x[k + 1] = std::exp((LD)t[k + 1]);
  }
  for (int o = 0; o < S.sh.n2; o++, k += 3) {
    const LD x1 = std::exp((LD)t[k]), x2 = std::exp((LD)t[k + 1]), Z = x1 + x2 + 1;
    x[k] = x1 / Z;
    x[k + 1] = x2 / Z;
    x[k + 2] = std::exp((LD)t[k + 2]);
  }
  LD Fl[64], Jl[64][40], r[64], dx[40];
  for (int it = 0; it < 8; it++) {
    eval_nat(S, x, Fl, Jl);
    for (int e = 0; e < S.ne; e++) r[e] = 1 - Fl[e];
    if (!solve<LD>(S.nu, Jl, r, dx)) return false;
    for (int j = 0; j < S.nu; j++) x[j] += dx[j];
  }
  eval_nat(S, x, Fl, Jl);
  for (int e = 0; e < S.ne; e++)
    if (!(std::fabs(Fl[e] - 1) < 1e-16L)) return false;
  return true;
}

// canonical form: S21 orbits by a ascending; S111 orbits with a < b < c, by (a, b)
void canonical(const System &S, LD *x) {
  int k = S.sh.n0;
  std::vector<std::pair<LD, LD>> s21;
  for (int o = 0; o < S.sh.n1; o++) s21.push_back({x[k + 2 * o], x[k + 2 * o + 1]});
  std::sort(s21.begin(), s21.end());
  for (int o = 0; o < S.sh.n1; o++) x[k + 2 * o] = s21[o].first, x[k + 2 * o + 1] = s21[o].second;
  k += 2 * S.sh.n1;
  std::vector<std::vector<LD>> s111;
  for (int o = 0; o < S.sh.n2; o++) {
    LD l[3] = {x[k + 3 * o], x[k + 3 * o + 1], 1 - x[k + 3 * o] - x[k + 3 * o + 1]};
    std::sort(l, l + 3);
    s111.push_back({l[0], l[1], x[k + 3 * o + 2]});
  }
  std::sort(s111.begin(), s111.end());
  for (int o = 0; o < S.sh.n2; o++)
    for (int q = 0; q < 3; q++) x[k + 3 * o + q] = s111[o][q];
}

LD min_bary(const System &S, const LD *x) {
  LD mb = 1.0L / 3;
  int k = S.sh.n0;
  for (int o = 0; o < S.sh.n1; o++, k += 2) mb = std::min(mb, std::min(x[k], 1 - 2 * x[k]));
  for (int o = 0; o < S.sh.n2; o++, k += 3) mb = std::min(mb, std::min(std::min(x[k], x[k + 1]), 1 - x[k] - x[k + 1]));
  return mb;
}

}  // namespace

int main() {
  std::printf("// Fully symmetric positive-interior triangle rules of degree 2p for the\n"
              "// prism rules of Table 1 (written by tri_rules_gen.cpp; see there).\n"
              "// Per degree p: orbit counts n0, n1, n2 and the parameters of the orbits:\n"
              "//   centroid: w;  S21: a, w  (points (a, a, 1-2a));  S111: a, b, w  (a < b < 1-a-b);\n"
              "// barycentric coordinates (l0, l1, l2), reference triangle area 1/2.\n");
  for (int p = 1; p <= 7; p++) {
    const System S(2 * p);
    std::vector<std::vector<LD>> sols;
#pragma omp parallel for schedule(dynamic, 16)
    for (long tr = 0; tr < kTrials[p]; tr++) {
      LD x[40];
      uint64_t seed = 0x1310119100000000ull + (uint64_t)p * 0x10000000ull + (uint64_t)tr;
      splitmix(seed);
      if (!path(S, seed, x)) continue;
      canonical(S, x);
      if (!(min_bary(S, x) > 1e-9L)) continue;
#pragma omp critical
      {
        bool dup = false;
        for (auto &s : sols) {
          LD dmax = 0;
          for (int j = 0; j < S.nu; j++) dmax = std::max(dmax, std::fabs(s[j] - x[j]));
          if (dmax < 1e-10L) dup = true;
        }
        if (!dup) sols.push_back(std::vector<LD>(x, x + S.nu));
      }
    }
    std::sort(sols.begin(), sols.end(),
              [&](const std::vector<LD> &u, const std::vector<LD> &v) { return min_bary(S, u.data()) > min_bary(S, v.data()); });
    std::printf("// p = %d (degree %d, %d points): %zu distinct PI rules in %ld paths; smallest barycentric "
                "coordinate of each:", p, 2 * p, S.sh.n0 + 3 * S.sh.n1 + 6 * S.sh.n2, sols.size(), kTrials[p]);
    for (auto &s : sols) std::printf(" %.6Lf", min_bary(S, s.data()));
    std::printf("\n{%d, %d, %d, %d, {", p, S.sh.n0, S.sh.n1, S.sh.n2);
    if (!sols.empty())
      for (int j = 0; j < S.nu; j++) std::printf("%s%.21Le", j ? ", " : "", sols[0][j]);
    std::printf("}},\n");
  }
  return 0;
}
