// Host side of ftlm_system_create: argument validation and the coupling
// tables of the Hamiltonian of Eq. (3) (Sec. II.A of arxiv 2607.25585),
// expressed in the ladder operators s+, s-, s^z that the row-gather kernels
// evaluate on the fly.
//
// For a vector u, u.s = u_z s^z + a s+ + conj(a) s-, a = (u_x - i u_y)/2
// (from s^x = (s+ + s-)/2, s^y = (s+ - s-)/(2i)).  A bilinear s_i^T A s_j
// then has the coefficients
//   s^z s^z : A_zz
//   s+ s-   : (A_xx + A_yy + i (A_xy - A_yx)) / 4       s- s+ : its conjugate
//   s+ s+   : (A_xx - A_yy - i (A_xy + A_yx)) / 4       s- s- : its conjugate
//   s+ s^z  : (A_xz - i A_yz) / 2                        s- s^z: its conjugate
//   s^z s+  : (A_zx - i A_zy) / 2                        s^z s-: its conjugate
// (the conjugate pairs hold because A is real).
#include <cmath>
#include <cstring>

#include "ftlm_internal.h"

namespace ftlm {

TabLayout make_layout(int n, int qmax) {
  TabLayout L;
  L.n = n;
  L.qmax = qmax;
  int o = 0;
  auto take = [&](int k) {
    int r = o;
    o += k;
    o = (o + 3) & ~3;  // keep 16-byte alignment for float tables
    return r;
  };
  L.off_m = take(n * qmax);
  L.off_up1 = take(n * qmax);
  L.off_dn1 = take(n * qmax);
  L.off_up2 = take(n * qmax);
  L.off_dn2 = take(n * qmax);
  L.off_iondiag = take(n * qmax);
  L.off_zz = take(n * n);
  L.off_pm = take(2 * n * n);
  L.off_pp = take(2 * n * n);
  L.off_rho = take(2 * n * n);
  L.off_hp = take(2 * n);
  L.off_bz = take(2 * n);
  L.off_bb = take(2 * n);
  L.off_hz = take(n);
  L.off_site4 = take(4 * n * qmax);
  L.off_pair4 = take(4 * n * n);
  L.total = o;
  return L;
}

void observable_coefs(const HostSystem& hs, const double* u_in, double out[3]) {
  double u[3] = {hs.Bdir[0], hs.Bdir[1], hs.Bdir[2]};
  if (u_in) {
    double nn = std::sqrt(u_in[0] * u_in[0] + u_in[1] * u_in[1] + u_in[2] * u_in[2]);
    if (nn > 0)
      for (int k = 0; k < 3; ++k) u[k] = u_in[k] / nn;
  }
  out[0] = u[2];
  out[1] = 0.5 * u[0];
  out[2] = -0.5 * u[1];
}

ftlm_status build_host_system(int n, const int* two_s, const double* J, const double* d_ion,
                              const double* e_axes, double g, const double B[3], const double* pos,
                              const ftlm_constants* k, HostSystem& hs, std::string& msg) {
  if (n < 1 || n > kMaxSites) {
    msg = "n_sites must be in 1.." + std::to_string(kMaxSites);
    return FTLM_ERR_INVALID_ARG;
  }
  if (!two_s || !B) {
    msg = "two_s and B must not be NULL";
    return FTLM_ERR_INVALID_ARG;
  }
  if (d_ion && !e_axes) {
    msg = "e_axes must be given when d_ion is";
    return FTLM_ERR_INVALID_ARG;
  }
  if (!std::isfinite(g)) {
    msg = "g must be finite";
    return FTLM_ERR_INVALID_ARG;
  }
  const double mu_B = k ? k->mu_B : 0.6717;
  const double C_dip = k ? k->C_dip : 0.6228;
  if (!std::isfinite(mu_B) || !std::isfinite(C_dip)) {
    msg = "constants must be finite";
    return FTLM_ERR_INVALID_ARG;
  }
  hs = HostSystem();
  hs.n = n;
  hs.two_s.assign(two_s, two_s + n);
  hs.q.resize(n);
  hs.stride.resize(n);
  uint64_t dim = 1;
  int qmax = 0;
  bool all_half = true;
  for (int i = 0; i < n; ++i) {
    if (two_s[i] < 1 || two_s[i] > kMaxQ - 1) {
      msg = "two_s[" + std::to_string(i) + "] must be in 1..15";
      return FTLM_ERR_INVALID_ARG;
    }
    hs.q[i] = two_s[i] + 1;
    hs.stride[i] = (int64_t)dim;
    dim *= (uint64_t)hs.q[i];
    if (dim > kMaxDim) {
      msg = "Hilbert-space dimension exceeds 2^36";
      return FTLM_ERR_UNSUPPORTED;
    }
    qmax = std::max(qmax, hs.q[i]);
    all_half = all_half && two_s[i] == 1;
  }
  hs.dim = dim;
  hs.qmax = qmax;
  hs.all_half = all_half;
  hs.g = g;
  double bn = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(B[a])) {
      msg = "B must be finite";
      return FTLM_ERR_INVALID_ARG;
    }
    hs.B[a] = B[a];
    bn += B[a] * B[a];
  }
  bn = std::sqrt(bn);
  if (bn > 0)
    for (int a = 0; a < 3; ++a) hs.Bdir[a] = B[a] / bn;

  // pair tensors A_ij (i<j): 2 J_ij I + C_dip g^2 / r^3 (I - 3 e e^T)
  std::vector<double> A((size_t)n * n * 9, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double* a = &A[((size_t)i * n + j) * 9];
      const double jij = J ? J[(size_t)i * n + j] : 0.0;
      if (!std::isfinite(jij)) {
        msg = "J must be finite";
        return FTLM_ERR_INVALID_ARG;
      }
      a[0] += 2.0 * jij;
      a[4] += 2.0 * jij;
      a[8] += 2.0 * jij;
      if (pos) {
        double r[3], r2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          r[c] = pos[3 * j + c] - pos[3 * i + c];
          r2 += r[c] * r[c];
        }
        if (!(r2 > 0.0) || !std::isfinite(r2)) {
          msg = "sites " + std::to_string(i) + " and " + std::to_string(j) + " coincide (or positions not finite)";
          return FTLM_ERR_INVALID_ARG;
        }
        const double pref = C_dip * g * g / (r2 * std::sqrt(r2));
        for (int x = 0; x < 3; ++x)
          for (int y = 0; y < 3; ++y) a[3 * x + y] += pref * ((x == y ? 1.0 : 0.0) - 3.0 * r[x] * r[y] / r2);
      }
    }

  hs.lay = make_layout(n, qmax);
  const TabLayout& L = hs.lay;
  std::vector<double>& t = hs.tab;
  t.assign(L.total, 0.0);
  for (int i = 0; i < n; ++i) {
    const double s = 0.5 * two_s[i];
    const double ss1 = s * (s + 1.0);
    // single-ion tensor d e e^T with a unit axis
    double di = d_ion ? d_ion[i] : 0.0, e[3] = {0, 0, 0};
    if (!std::isfinite(di)) {
      msg = "d_ion must be finite";
      return FTLM_ERR_INVALID_ARG;
    }
    if (di != 0.0) {
      double en = std::sqrt(e_axes[3 * i] * e_axes[3 * i] + e_axes[3 * i + 1] * e_axes[3 * i + 1] +
                            e_axes[3 * i + 2] * e_axes[3 * i + 2]);
      if (!(en > 0.0) || !std::isfinite(en)) {
        msg = "e_axes[" + std::to_string(i) + "] must be a nonzero finite vector where d_ion != 0";
        return FTLM_ERR_INVALID_ARG;
      }
      for (int c = 0; c < 3; ++c) e[c] = e_axes[3 * i + c] / en;
    }
    // b = (e_x - i e_y)/2;  d (e.s)^2 = d [e_z^2 s_z^2 + |b|^2 (s+s- + s-s+) + e_z b (s_z s+ + s+ s_z) + h.c. + b^2 s+^2 + h.c.]
    const double ez2 = e[2] * e[2], bb_abs2 = 0.25 * (e[0] * e[0] + e[1] * e[1]);
    for (int a = 0; a < hs.q[i]; ++a) {
      const double m = a - s;
      t[L.off_m + i * qmax + a] = m;
      t[L.off_up1 + i * qmax + a] = a >= 1 ? std::sqrt(ss1 - (m - 1.0) * m) : 0.0;
      t[L.off_dn1 + i * qmax + a] = a + 1 < hs.q[i] ? std::sqrt(ss1 - (m + 1.0) * m) : 0.0;
      t[L.off_iondiag + i * qmax + a] = di * (ez2 * m * m + bb_abs2 * 2.0 * (ss1 - m * m));
    }
    for (int a = 0; a < hs.q[i]; ++a) {
      t[L.off_up2 + i * qmax + a] =
          a >= 2 ? t[L.off_up1 + i * qmax + a] * t[L.off_up1 + i * qmax + a - 1] : 0.0;
      t[L.off_dn2 + i * qmax + a] =
          a + 2 < hs.q[i] ? t[L.off_dn1 + i * qmax + a] * t[L.off_dn1 + i * qmax + a + 1] : 0.0;
    }
    // d e_z b and d b^2
    t[L.off_bz + 2 * i] = di * e[2] * 0.5 * e[0];
    t[L.off_bz + 2 * i + 1] = -di * e[2] * 0.5 * e[1];
    t[L.off_bb + 2 * i] = di * 0.25 * (e[0] * e[0] - e[1] * e[1]);
    t[L.off_bb + 2 * i + 1] = -di * 0.5 * e[0] * e[1];
    // Zeeman mu_B g B.s: s^z coefficient h_z, s+ coefficient (h_x - i h_y)/2
    const double h[3] = {mu_B * g * B[0], mu_B * g * B[1], mu_B * g * B[2]};
    t[L.off_hz + i] = h[2];
    t[L.off_hp + 2 * i] = 0.5 * h[0];
    t[L.off_hp + 2 * i + 1] = -0.5 * h[1];
  }
  bool real_pm = true;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double* a = &A[((size_t)i * n + j) * 9];
      const double xx = a[0], xy = a[1], xz = a[2], yx = a[3], yy = a[4], yz = a[5], zx = a[6], zy = a[7],
                   zz = a[8];
      const int ij = i * n + j, ji = j * n + i;
      t[L.off_zz + ij] = zz;
      t[L.off_pm + 2 * ij] = 0.25 * (xx + yy);
      t[L.off_pm + 2 * ij + 1] = 0.25 * (xy - yx);
      t[L.off_pp + 2 * ij] = 0.25 * (xx - yy);
      t[L.off_pp + 2 * ij + 1] = -0.25 * (xy + yx);
      // s+_i s^z_j and s^z_i s+_j (= s+_j s^z_i, stored under the ordered pair (j, i))
      t[L.off_rho + 2 * ij] = 0.5 * xz;
      t[L.off_rho + 2 * ij + 1] = -0.5 * yz;
      t[L.off_rho + 2 * ji] = 0.5 * zx;
      t[L.off_rho + 2 * ji + 1] = -0.5 * zy;
      if (t[L.off_pm + 2 * ij + 1] != 0.0) real_pm = false;
    }
  hs.real_pm = real_pm;
  // the packed copies
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < qmax; ++a) {
      double* q4 = &t[L.off_site4 + 4 * (i * qmax + a)];
      q4[0] = t[L.off_up1 + i * qmax + a];
      q4[1] = t[L.off_dn1 + i * qmax + a];
      q4[2] = t[L.off_m + i * qmax + a];
      q4[3] = t[L.off_iondiag + i * qmax + a];
    }
  for (int ij = 0; ij < n * n; ++ij) {
    double* p4 = &t[L.off_pair4 + 4 * ij];
    p4[0] = t[L.off_pm + 2 * ij];
    p4[1] = t[L.off_pm + 2 * ij + 1];
    p4[2] = t[L.off_pp + 2 * ij];
    p4[3] = t[L.off_pp + 2 * ij + 1];
  }
  return FTLM_OK;
}

}  // namespace ftlm
