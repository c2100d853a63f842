"""The 1D factor tables behind the operator apply's sum factorisation
(build_sf_tables in csrc/fem_tables.cpp), checked on the host: a small C++
driver compiled against the library's table builder multiplies the factors
back together and compares every entry of the full prism table (value and the
three reference derivatives at every point, every DOF, p = 1..7)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1310_1191_gb300", "csrc")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include "fem_internal.h"
using namespace fem;
int main() {
  for (int p = 1; p <= 7; p++) {
    HostRule r;
    if (!build_host_rule(FEM_PRISM6, p, &r)) return 2;
    std::vector<double> f;
    build_sf_tables(p, f);
    const int n = p + 1, nt = n * (n + 1) / 2, np_ = n | 1, ns = r.ns, nab = n * n;
    if ((int)f.size() != 5 * n * n + 3 * nt * np_) return 3;
    const double *Pa = f.data(), *Px = Pa + n * n, *Pe = Px + n * n, *Bq = Pe + n * n,
                 *Bx = Bq + nt * np_, *By = Bx + nt * np_, *L = By + nt * np_, *dL = L + n * n;
    int ti[64];
    for (int m = 0, t = 0; m < n; m++)
      for (int i = m; i >= 0; i--, t++) ti[t] = i;
    double err = 0.0, mx[4] = {0, 0, 0, 0}, e4[4] = {0, 0, 0, 0};
    for (int iz = 0; iz < n; iz++)
      for (int ia = 0; ia < n; ia++)
        for (int ib = 0; ib < n; ib++) {
          const int q = iz * nab + ia * n + ib;
          for (int k = 0; k < n; k++)
            for (int t = 0; t < nt; t++) {
              const int i = ti[t];
              const double *ph = &r.phi[(size_t)4 * q * ns + t + nt * k];
              const double v[4] = {
                  Pa[ia * n + i] * Bq[t * np_ + ib] * L[iz * n + k],
                  Px[ia * n + i] * Bx[t * np_ + ib] * L[iz * n + k],
                  (Pe[ia * n + i] * Bx[t * np_ + ib] + Pa[ia * n + i] * By[t * np_ + ib]) * L[iz * n + k],
                  Pa[ia * n + i] * Bq[t * np_ + ib] * dL[iz * n + k]};
              for (int d = 0; d < 4; d++) {
                e4[d] = std::fmax(e4[d], std::fabs(v[d] - ph[(size_t)d * ns]));
                mx[d] = std::fmax(mx[d], std::fabs(ph[(size_t)d * ns]));
              }
            }
        }
    for (int d = 0; d < 4; d++) err = std::fmax(err, e4[d] / mx[d]);
    printf("%d %.3e\n", p, err);
  }
  return 0;
}
"""


def test_factor_tables_rebuild_the_prism_table(tmp_path):
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "sf_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "sf_check"
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           "-I", inc, str(src), os.path.join(CSRC, "fem_tables.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    errs = {int(p): float(e) for p, e in zip(out[0::2], out[1::2])}
    assert sorted(errs) == list(range(1, 8))
    # products of 1D factors vs entries built in one piece: a few ulps
    assert max(errs.values()) < 1e-13, errs
