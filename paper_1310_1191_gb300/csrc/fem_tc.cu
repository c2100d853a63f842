// Host side of the tensor-core path: the launch dispatcher (argument
// marshalling, choice of the instantiation by precision, form and rule) and
// the Phi^T operand images.  The kernel is in fem_tc.cuh, its instantiations
// in fem_tc_*.cu.
#include "fem_tc.cuh"

namespace fem {

int launch_tc(int p, bool f16, const DevTable &d, const TcLaunch &l, void *stream) {
  TcArgs a;
  a.n = l.n;
  a.coords = l.coords;
  a.coeffs = l.coeffs;
  a.cstride = l.cstride;
  a.qp = d.qp;
  a.phiq = d.phiq32;
  a.img = f16 ? d.img_f16 : d.img_bf16;
  a.phimax = d.phimax;
  a.aphi = f16 ? d.aphi_f16 : 0;
  a.A = l.A;
  a.b = l.b;
  a.status = l.status;
  a.layout = l.layout;
  a.err = l.err;
  a.stall = l.stall;
  a.perm = l.perm;
  a.offA = l.offA;
  a.offb = l.offb;
  a.ucoef = l.ucoef;
  a.phiT = d.phiT32;
  a.mlpw = l.mlpw;
  a.mlpw2 = l.mlpw2;
  for (int i = 0; i < 4; i++) {
    a.nrm[i] = l.nrm[i];
    a.box[i] = l.box[i];
  }
  a.law_iters = l.law_iters;
  a.hw_tanh = l.hw_tanh;
  a.limA = l.limA;
  a.limb = l.limb;
  a.nmesh = l.nmesh;
  if (l.elastic && (a.perm || a.offA || a.offb)) {
    set_error("tensor-core elasticity takes dense outputs only");
    return FEM_EINVAL;
  }
  if (!a.img) {
    set_error("tensor-core tables missing for this degree");
    return FEM_EUNSUPPORTED;
  }
  if (l.elastic)
    return d.rule == FEM_RULE_TABLE1 ? launch_tc_elastic_t1(p, f16, a, stream) : launch_tc_elastic(p, f16, a, stream);
  if (l.law != 0) {
    if (f16 || !a.ucoef || (l.law == 2 && (!a.mlpw || !a.mlpw2))) {
      set_error("tensor-core law integration: BF16x3 with field coefficients (and a network) only");
      return FEM_EINVAL;
    }
    if (d.rule != FEM_RULE_COLLAPSED) {
      set_error("tensor-core law integration: collapsed-rule tables only");
      return FEM_EUNSUPPORTED;
    }
    return launch_tc_law(p, l.law, a, stream);
  }
  if (d.rule == FEM_RULE_TABLE1) return launch_tc_scalar_t1(p, f16, a, stream);
  return f16 ? launch_tc_scalar_f16(p, a, stream) : launch_tc_scalar_bf16(p, a, stream);
}

// Image of Phi^T for the B operand: per K chunk of 32, [hi | lo] blocks of
// NP x 32 16-bit values in the canonical K-major core-matrix layout
// (8 rows x 8 values = 128 bytes per core matrix; K-adjacent core matrices
// 128 bytes apart, 8-row groups (KC/8)*128 bytes apart).  Rows i >= NS and
// k >= 4 NQ are zero.
template <int P, int RULE>
static void build_image_p(const std::vector<double> &phi, bool f16, int aphi, std::vector<uint16_t> &out) {
  using C = TcCfg<P, false, 0, RULE>;
  out.assign((size_t)C::NCH * 2 * C::NP * C::KC, 0);
  const double scale = std::ldexp(1.0, aphi);
  for (int c = 0; c < C::NCH; c++) {
    uint16_t *hi = out.data() + (size_t)c * 2 * C::NP * C::KC;
    uint16_t *lo = hi + (size_t)C::NP * C::KC;
    for (int i = 0; i < C::NS; i++)
      for (int kl = 0; kl < C::KC; kl++) {
        const int k = c * C::KC + kl;
        if (k >= 4 * C::NQ) continue;
        const double x = phi[(size_t)k * C::NS + i] * scale;
        uint16_t h, l;
        if (f16) {
          __half hh = __double2half((double)x);
          h = __half_as_ushort(hh);
          l = __half_as_ushort(__double2half(x - (double)__half2float(hh)));
        } else {
          __nv_bfloat16 hh = __double2bfloat16(x);
          h = __bfloat16_as_ushort(hh);
          l = __bfloat16_as_ushort(__double2bfloat16(x - (double)__bfloat162float(hh)));
        }
        const size_t off = ((size_t)(i >> 3) * (C::KC / 8) + (kl >> 3)) * 64 + (i & 7) * 8 + (kl & 7);
        hi[off] = h;
        lo[off] = l;
      }
  }
}

void build_tc_image(int p, int rule, const std::vector<double> &phi, bool f16, int aphi, std::vector<uint16_t> &out) {
  if (rule == FEM_RULE_TABLE1) {
    switch (p) {
      case 1: build_image_p<1, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 2: build_image_p<2, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 3: build_image_p<3, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 4: build_image_p<4, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 5: build_image_p<5, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 6: build_image_p<6, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
      case 7: build_image_p<7, FEM_RULE_TABLE1>(phi, f16, aphi, out); break;
    }
    return;
  }
  switch (p) {
    case 1: build_image_p<1, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 2: build_image_p<2, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 3: build_image_p<3, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 4: build_image_p<4, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 5: build_image_p<5, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 6: build_image_p<6, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
    case 7: build_image_p<7, FEM_RULE_COLLAPSED>(phi, f16, aphi, out); break;
  }
}

}  // namespace fem
