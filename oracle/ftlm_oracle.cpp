// Plain CPU FP64 oracle for the finite-temperature Lanczos method (FTLM) on
// anisotropic spin Hamiltonians.  TEST INFRASTRUCTURE ONLY: the tests, the
// smoke check and the CPU-baseline leg of the benchmark call it; the product
// path never does.  It shares no code with the CUDA library.
//
// What it follows (arxiv 2607.25585, Schnack, "Finite-temperature Lanczos for
// anisotropic spin systems using triple-hybrid HPC"):
//   * the Hamiltonian of Eq. (3) (Sec. II.A): Heisenberg exchange 2 J_ij s_i.s_j
//     over i<j, single-ion d_i (s_i.e_i)^2, Zeeman mu_B g B.s_i, and the
//     all-pairs dipolar term (mu0 mu_B^2 / 4 pi) g^2 / r^3 (s_i.s_j - 3 (s_i.e)(e.s_j));
//   * the product basis of dimension prod_i (2 s_i + 1) (Sec. II.A);
//   * random start vectors with Gaussian complex components, Eq. (2), used in
//     the trace estimator Eq. (1) with the d / R prefactor of Eq. (5);
//   * the Lanczos recurrence with two predecessor vectors and optional full
//     re-orthogonalisation (Sec. II.C);
//   * the FTLM estimators Eq. (4) (observable ratio, same r in numerator and
//     denominator) and Eq. (5) (partition function, Gamma = 1: no symmetry);
//   * symmetric FTLM (sFTLM), Eqs. (E-2-G) and (E-2-H): the observable
//     between the two halves of e^{-beta H}, with <m|O|n> from the matrix of
//     O in the Lanczos basis;
//   * pairs of mutually time-reversed random vectors (Sec. II.B: the
//     time-reversal symmetry used for the FTLM approximation, tau = 1 in the
//     figures of Sec. III), Theta = exp(-i pi S^y) K with K the complex
//     conjugation in the S^z product basis.
//
// Readings where the paper is silent (this oracle and the CUDA library both take them):
//   basis index mu = sum_i a_i * prod_{k<i} q_k, site 0 least significant,
//   digit a_i = m_i + s_i;  random numbers: Philox4x32-10 (Salmon et al.,
//   SC'11) + Box-Muller;  each r normalised to 1;  Z returned as ln Z with the
//   lowest Ritz value E0 factored out;  M_B = -g <B^.S> in units of mu_B.
//
// Pins (tests/test_oracle_*.py) tie every function to closed forms, the dense
// definition, LAPACK and exact limits.  A finite-R FTLM estimate differs from
// the exact thermodynamics by a statistical error, so at finite R it is pinned
// only through its exact limits (all basis vectors as start vectors; full
// Krylov depth, where it equals the stochastic trace of Eq. 1): parity
// unpinned at tolerance level for finite R against exact diagonalisation.
//
// Everything is double precision and deliberately unoptimised: the matvec is a
// column scatter (for each source state nu, apply every term of H to |nu>),
// the tridiagonal eigenproblem is solved by cyclic Jacobi on the dense matrix.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

extern "C" {

typedef struct {
  int n;                 // number of sites
  const int* two_s;      // [n] twice the spin quantum number (1 = spin 1/2)
  const double* J;       // [n*n] row-major exchange in K; J[i*n+j], i<j, is used
  const double* d_ion;   // [n] single-ion strength in K, or NULL (= 0)
  const double* e_axes;  // [n*3] single-ion axes (normalised here), or NULL
  double g;              // g factor (Zeeman g_i = g, dipolar g^2)
  const double* B;       // [3] field in Tesla
  const double* pos;     // [n*3] positions in Angstrom, or NULL = no dipolar term
  double mu_B;           // Bohr magneton in K/T
  double C_dip;          // mu0 mu_B^2 / (4 pi k_B) in K Angstrom^3
} oracle_system;

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Model (Eq. 3): pair tensors, site fields, single-ion tensors.
// ---------------------------------------------------------------------------
struct Model {
  int n = 0;
  std::vector<int> two_s;
  std::vector<int64_t> q, stride;
  int64_t dim = 1;
  // A[(i*n+j)*9 + 3a+b] = coefficient of s_i^a s_j^b for i<j (a,b in x,y,z)
  std::vector<double> A;
  // single-ion: D[i*9 + 3a+b] = d_i e_a e_b  (coefficient of s_i^a s_i^b)
  std::vector<double> D;
  double h[3] = {0, 0, 0};  // mu_B g B, the Zeeman field in K
  double g = 2.0;
  double Bdir[3] = {0, 0, 1};
};

bool build_model(const oracle_system* s, Model& m) {
  if (!s || s->n <= 0 || !s->two_s || !s->B) return false;
  m.n = s->n;
  m.two_s.assign(s->two_s, s->two_s + s->n);
  m.q.resize(m.n);
  m.stride.resize(m.n);
  m.dim = 1;
  for (int i = 0; i < m.n; ++i) {
    if (m.two_s[i] < 1) return false;
    m.q[i] = m.two_s[i] + 1;
    m.stride[i] = m.dim;
    m.dim *= m.q[i];
  }
  const int n = m.n;
  m.A.assign((size_t)n * n * 9, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      double* a = &m.A[((size_t)i * n + j) * 9];
      // Heisenberg exchange: 2 J_ij s_i . s_j
      double jij = s->J ? s->J[(size_t)i * n + j] : 0.0;
      for (int k = 0; k < 3; ++k) a[4 * k] += 2.0 * jij;
      // dipolar: C_dip g^2 / r^3 (s_i.s_j - 3 (s_i.e)(e.s_j)), e = unit(pos_j - pos_i)
      if (s->pos) {
        double r[3], r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
          r[k] = s->pos[3 * j + k] - s->pos[3 * i + k];
          r2 += r[k] * r[k];
        }
        if (r2 <= 0.0) return false;  // coincident sites
        double rr = std::sqrt(r2);
        double pref = s->C_dip * s->g * s->g / (r2 * rr);
        for (int a1 = 0; a1 < 3; ++a1)
          for (int b1 = 0; b1 < 3; ++b1) {
            double e_ab = r[a1] * r[b1] / r2;
            a[3 * a1 + b1] += pref * ((a1 == b1 ? 1.0 : 0.0) - 3.0 * e_ab);
          }
      }
    }
  }
  m.D.assign((size_t)n * 9, 0.0);
  for (int i = 0; i < n; ++i) {
    double di = s->d_ion ? s->d_ion[i] : 0.0;
    if (di == 0.0) continue;
    if (!s->e_axes) return false;
    double e[3] = {s->e_axes[3 * i], s->e_axes[3 * i + 1], s->e_axes[3 * i + 2]};
    double en = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (en <= 0.0) return false;
    for (int k = 0; k < 3; ++k) e[k] /= en;
    for (int a1 = 0; a1 < 3; ++a1)
      for (int b1 = 0; b1 < 3; ++b1) m.D[(size_t)i * 9 + 3 * a1 + b1] = di * e[a1] * e[b1];
  }
  m.g = s->g;
  double bn = 0.0;
  for (int k = 0; k < 3; ++k) {
    m.h[k] = s->mu_B * s->g * s->B[k];
    bn += s->B[k] * s->B[k];
  }
  bn = std::sqrt(bn);
  if (bn > 0.0)
    for (int k = 0; k < 3; ++k) m.Bdir[k] = s->B[k] / bn;
  return true;
}

// ---------------------------------------------------------------------------
// Ladder form of the operators (derived from s^x = (s+ + s-)/2,
// s^y = (s+ - s-)/(2i)).  For a vector u, u.s = u_z s^z + a s+ + conj(a) s-,
// with a = (u_x - i u_y)/2.  For a bilinear s_i^T A s_j the coefficients of
// the ladder products follow by substituting both expansions.
// ---------------------------------------------------------------------------
struct PairLadder {
  double zz;
  cplx pm, mp, pp, mm, pz, mz, zp, zm;  // p = s+, m = s-, z = s^z; first letter site i
};

PairLadder pair_ladder(const double* A) {
  const double xx = A[0], xy = A[1], xz = A[2], yx = A[3], yy = A[4], yz = A[5], zx = A[6],
               zy = A[7], zz = A[8];
  const cplx I(0.0, 1.0);
  PairLadder L;
  L.zz = zz;
  L.pm = 0.25 * (xx + yy + I * (xy - yx));
  L.mp = 0.25 * (xx + yy - I * (xy - yx));
  L.pp = 0.25 * (xx - yy - I * (xy + yx));
  L.mm = 0.25 * (xx - yy + I * (xy + yx));
  L.pz = 0.5 * (xz - I * yz);
  L.mz = 0.5 * (xz + I * yz);
  L.zp = 0.5 * (zx - I * zy);
  L.zm = 0.5 * (zx + I * zy);
  return L;
}

// <m+1| s+ |m> and <m-1| s- |m>
inline double cplus(double s, double m) { return std::sqrt(std::max(0.0, s * (s + 1.0) - m * (m + 1.0))); }
inline double cminus(double s, double m) { return std::sqrt(std::max(0.0, s * (s + 1.0) - m * (m - 1.0))); }

// One column of H: all (row, value) with H[row][nu] != 0, obtained by applying
// every term of Eq. (3) to the basis state |nu>.  Entries may repeat a row.
struct Entry {
  int64_t row;
  cplx val;
};

void column_entries(const Model& M, const std::vector<PairLadder>& PL, int64_t nu,
                    std::vector<Entry>& out) {
  out.clear();
  const int n = M.n;
  std::vector<double> s(n), m(n);
  int64_t rem = nu;
  for (int i = 0; i < n; ++i) {
    int64_t a = rem % M.q[i];
    rem /= M.q[i];
    s[i] = 0.5 * M.two_s[i];
    m[i] = (double)a - s[i];
  }
  cplx diag = 0.0;
  // pair terms
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      const PairLadder& L = PL[(size_t)i * n + j];
      const bool ui = m[i] < s[i], di = m[i] > -s[i];
      const bool uj = m[j] < s[j], dj = m[j] > -s[j];
      const int64_t si = M.stride[i], sj = M.stride[j];
      diag += L.zz * m[i] * m[j];
      if (ui && dj) out.push_back({nu + si - sj, L.pm * cplus(s[i], m[i]) * cminus(s[j], m[j])});
      if (di && uj) out.push_back({nu - si + sj, L.mp * cminus(s[i], m[i]) * cplus(s[j], m[j])});
      if (ui && uj) out.push_back({nu + si + sj, L.pp * cplus(s[i], m[i]) * cplus(s[j], m[j])});
      if (di && dj) out.push_back({nu - si - sj, L.mm * cminus(s[i], m[i]) * cminus(s[j], m[j])});
      if (ui) out.push_back({nu + si, L.pz * cplus(s[i], m[i]) * m[j]});
      if (di) out.push_back({nu - si, L.mz * cminus(s[i], m[i]) * m[j]});
      if (uj) out.push_back({nu + sj, L.zp * m[i] * cplus(s[j], m[j])});
      if (dj) out.push_back({nu - sj, L.zm * m[i] * cminus(s[j], m[j])});
    }
  }
  // single-site terms: Zeeman h.s_i and single-ion s_i^T D_i s_i
  const cplx I(0.0, 1.0);
  for (int i = 0; i < n; ++i) {
    const double si = s[i], mi = m[i];
    const int64_t st = M.stride[i];
    const bool up = mi < si, dn = mi > -si;
    // Zeeman: h_z s^z + a s+ + conj(a) s-, a = (h_x - i h_y)/2
    const cplx ah = 0.5 * (M.h[0] - I * M.h[1]);
    diag += M.h[2] * mi;
    if (up) out.push_back({nu + st, ah * cplus(si, mi)});
    if (dn) out.push_back({nu - st, std::conj(ah) * cminus(si, mi)});
    // single-ion, D = d e e^T: d (e.s)^2 = d (e_z s^z + b s+ + conj(b) s-)^2, b = (e_x - i e_y)/2
    const double* D = &M.D[(size_t)i * 9];
    const double dd = D[0] + D[4] + D[8];  // = d_i (trace of d e e^T, |e| = 1)
    if (dd != 0.0) {
      // recover d e_a e_b products: ez2 = D_zz, |b|^2 d = (D_xx + D_yy)/4, etc.
      const double dzz = D[8];
      const cplx bz = 0.5 * (D[2] - I * D[5]);                      // d e_z b
      const cplx bb = 0.25 * (D[0] - D[4] - I * (D[1] + D[3]));     // d b^2
      const double bbar = 0.25 * (D[0] + D[4]);                     // d |b|^2
      // diagonal: d [e_z^2 m^2 + |b|^2 (s+s- + s-s+)] = dzz m^2 + bbar * 2 (s(s+1) - m^2)
      diag += dzz * mi * mi + bbar * 2.0 * (si * (si + 1.0) - mi * mi);
      // +1: d e_z b (s^z s+ + s+ s^z) |m> = d e_z b (2m + 1) c+(m) |m+1>
      if (up) out.push_back({nu + st, bz * (2.0 * mi + 1.0) * cplus(si, mi)});
      if (dn) out.push_back({nu - st, std::conj(bz) * (2.0 * mi - 1.0) * cminus(si, mi)});
      // +2: d b^2 s+ s+ |m> = d b^2 c+(m) c+(m+1) |m+2>
      if (mi + 1.0 < si) out.push_back({nu + 2 * st, bb * cplus(si, mi) * cplus(si, mi + 1.0)});
      if (mi - 1.0 > -si)
        out.push_back({nu - 2 * st, std::conj(bb) * cminus(si, mi) * cminus(si, mi - 1.0)});
    }
  }
  out.push_back({nu, diag});
}

std::vector<PairLadder> all_pair_ladders(const Model& M) {
  std::vector<PairLadder> PL((size_t)M.n * M.n);
  for (int i = 0; i < M.n; ++i)
    for (int j = i + 1; j < M.n; ++j) PL[(size_t)i * M.n + j] = pair_ladder(&M.A[((size_t)i * M.n + j) * 9]);
  return PL;
}

// y = H x by column scatter, x and y [dim][nvec] complex.
void apply_h(const Model& M, const std::vector<PairLadder>& PL, const cplx* x, cplx* y, int64_t nvec) {
  std::fill(y, y + M.dim * nvec, cplx(0.0));
  std::vector<Entry> col;
  for (int64_t nu = 0; nu < M.dim; ++nu) {
    column_entries(M, PL, nu, col);
    for (const Entry& e : col)
      for (int64_t k = 0; k < nvec; ++k) y[e.row * nvec + k] += e.val * x[nu * nvec + k];
  }
}

// y = (u . S) x with S = sum_i s_i (one-body, column scatter).
void apply_sdir(const Model& M, const double* u, const cplx* x, cplx* y, int64_t nvec) {
  std::fill(y, y + M.dim * nvec, cplx(0.0));
  const cplx I(0.0, 1.0);
  const cplx a = 0.5 * (u[0] - I * u[1]);
  for (int64_t nu = 0; nu < M.dim; ++nu) {
    int64_t rem = nu;
    for (int i = 0; i < M.n; ++i) {
      int64_t ai = rem % M.q[i];
      rem /= M.q[i];
      double s = 0.5 * M.two_s[i], m = (double)ai - s;
      for (int64_t k = 0; k < nvec; ++k) {
        const cplx xv = x[nu * nvec + k];
        y[nu * nvec + k] += u[2] * m * xv;
        if (m < s) y[(nu + M.stride[i]) * nvec + k] += a * cplus(s, m) * xv;
        if (m > -s) y[(nu - M.stride[i]) * nvec + k] += std::conj(a) * cminus(s, m) * xv;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.
// ---------------------------------------------------------------------------
void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c[0];
    uint64_t p1 = (uint64_t)M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// 53-bit uniform in (0, 1] from two 32-bit words.
inline double uniform53(uint32_t hi, uint32_t lo) {
  uint64_t k = ((uint64_t)hi << 21) | ((uint64_t)lo >> 11);
  return ((double)k + 1.0) * (1.0 / 9007199254740992.0);
}

// Component nu of random vector number rg (global index): complex Gaussian,
// re and im independent N(0, 1).
cplx gaussian_component(uint64_t seed, uint64_t rg, uint64_t nu) {
  uint32_t ctr[4] = {(uint32_t)nu, (uint32_t)(nu >> 32), (uint32_t)rg, (uint32_t)(rg >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox(ctr, key, o);
  const double u1 = uniform53(o[0], o[1]);
  const double u2 = uniform53(o[2], o[3]);
  const double rho = std::sqrt(-2.0 * std::log(u1));
  const double ang = 2.0 * M_PI * u2;
  return cplx(rho * std::cos(ang), rho * std::sin(ang));
}

// ---------------------------------------------------------------------------
// Lanczos (Sec. II.C): three-term recurrence, optional full re-orthogonalisation.
// ---------------------------------------------------------------------------
cplx dot(const std::vector<cplx>& a, const std::vector<cplx>& b) {  // <a|b>
  cplx s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += std::conj(a[i]) * b[i];
  return s;
}

// v0 must be normalised.  alpha[M], beta[M] (beta[j] = norm after step j, the
// off-diagonal T[j][j+1]), p[M] = <v_j | u>, u = (dir.S) v0.
// keep: if given, receives the Lanczos vectors v_0 .. v_{M_eff-1}.
int lanczos(const Model& M, const std::vector<PairLadder>& PL, const std::vector<cplx>& v0, int maxM,
            int reorth, double tol, const double* dir, double* alpha, double* beta, cplx* p,
            std::vector<std::vector<cplx>>* keep = nullptr) {
  const int64_t d = M.dim;
  std::vector<cplx> u(d), w(d), vprev(d, 0.0), v = v0;
  apply_sdir(M, dir, v0.data(), u.data(), 1);
  std::vector<std::vector<cplx>> basis;
  if (reorth) basis.push_back(v);
  if (keep) keep->assign(1, v);
  double bj = 0.0, scale = 0.0;
  int meff = maxM;
  for (int j = 0; j < maxM; ++j) {
    apply_h(M, PL, v.data(), w.data(), 1);
    const double a = std::real(dot(v, w));
    alpha[j] = a;
    p[j] = dot(v, u);
    for (int64_t i = 0; i < d; ++i) w[i] -= a * v[i] + bj * vprev[i];
    if (reorth) {
      for (int pass = 0; pass < 2; ++pass)
        for (const auto& b : basis) {
          const cplx c = dot(b, w);
          for (int64_t i = 0; i < d; ++i) w[i] -= c * b[i];
        }
    }
    double nb = 0.0;
    for (int64_t i = 0; i < d; ++i) nb += std::norm(w[i]);
    nb = std::sqrt(nb);
    beta[j] = nb;
    scale = std::max(scale, std::max(std::fabs(a), bj));
    if (j == maxM - 1) break;
    if (nb <= tol * scale || (reorth && (int64_t)basis.size() >= d)) {
      meff = j + 1;
      break;
    }
    vprev = v;
    for (int64_t i = 0; i < d; ++i) v[i] = w[i] / nb;
    if (reorth) basis.push_back(v);
    if (keep) keep->push_back(v);
    bj = nb;
  }
  if (keep) keep->resize(meff);
  return meff;
}

// Cyclic Jacobi on the dense symmetric tridiagonal matrix T (alpha on the
// diagonal, beta[0..m-2] off the diagonal).  evecs[k*m + n] = U_{kn}.
void jacobi_tridiag(int m, const double* alpha, const double* beta, double* evals, double* evecs) {
  std::vector<double> a((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    a[(size_t)i * m + i] = alpha[i];
    if (i + 1 < m) a[(size_t)i * m + i + 1] = a[(size_t)(i + 1) * m + i] = beta[i];
  }
  std::vector<double> V((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  double fro = 0.0;
  for (double x : a) fro += x * x;
  // an off-diagonal element below this is treated as zero (absolute accuracy
  // of the eigenvalues ~1e-17 of the Frobenius norm)
  const double negligible = 1e-17 * std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int pp = 0; pp < m; ++pp)
      for (int qq = pp + 1; qq < m; ++qq) {
        const double apq = a[(size_t)pp * m + qq];
        if (std::fabs(apq) <= negligible) continue;
        ++rotated;
        const double app = a[(size_t)pp * m + pp], aqq = a[(size_t)qq * m + qq];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < m; ++r) {  // columns p, q
          const double arp = a[(size_t)r * m + pp], arq = a[(size_t)r * m + qq];
          a[(size_t)r * m + pp] = c * arp - s * arq;
          a[(size_t)r * m + qq] = s * arp + c * arq;
        }
        for (int r = 0; r < m; ++r) {  // rows p, q
          const double apr = a[(size_t)pp * m + r], aqr = a[(size_t)qq * m + r];
          a[(size_t)pp * m + r] = c * apr - s * aqr;
          a[(size_t)qq * m + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < m; ++r) {
          const double vrp = V[(size_t)r * m + pp], vrq = V[(size_t)r * m + qq];
          V[(size_t)r * m + pp] = c * vrp - s * vrq;
          V[(size_t)r * m + qq] = s * vrp + c * vrq;
        }
      }
    if (!rotated) break;
  }
  for (int i = 0; i < m; ++i) evals[i] = a[(size_t)i * m + i];
  std::memcpy(evecs, V.data(), sizeof(double) * (size_t)m * m);
}

// Time reversal Theta = exp(-i pi S^y) K on x (Sec. II.B).  On one site,
// exp(-i pi s^y)|s, m> = (-1)^(s - m) |s, -m>, so for a product state
// Theta |mu> = prod_i (-1)^(s_i - m_i) |mu'> with m_i -> -m_i, and the
// coefficient is conjugated: y[mu'] = prod_i (-1)^(s_i - m_i(mu)) conj(x[mu]).
void time_reverse(const Model& M, const cplx* x, cplx* y, int64_t nvec) {
  for (int64_t mu = 0; mu < M.dim; ++mu) {
    int64_t image = 0;
    int sign_exp = 0;
    for (int i = 0; i < M.n; ++i) {
      const int64_t a = (mu / M.stride[i]) % M.q[i];  // a = m + s
      const int64_t a_img = M.two_s[i] - a;          // m -> -m
      image += a_img * M.stride[i];
      sign_exp += (int)(M.two_s[i] - a);             // s - m = 2s - a
    }
    const double ph = (sign_exp % 2) ? -1.0 : 1.0;
    for (int64_t k = 0; k < nvec; ++k) y[image * nvec + k] = ph * std::conj(x[mu * nvec + k]);
  }
}

// Start vector number r of a run of R (Eq. 2 and the start modes): 0 = Philox
// random vector vec_offset + r, 1 = basis vector |basis_offset + r>, 2 = column
// r of the user block [d][R], 3 = time-reversed pairs (vector v = vec_offset + r
// is random vector v / 2, time-reversed when v is odd).  Normalised to 1.
bool start_vector(const Model& M, int r, int R, uint64_t seed, uint64_t vec_offset, int start_mode,
                  int64_t basis_offset, const double* user_start, std::vector<cplx>& v0) {
  v0.assign(M.dim, 0.0);
  auto normalise = [](std::vector<cplx>& v) {
    double nrm = 0.0;
    for (const auto& z : v) nrm += std::norm(z);
    nrm = std::sqrt(nrm);
    for (auto& z : v) z /= nrm;
  };
  if (start_mode == 0) {
    for (int64_t nu = 0; nu < M.dim; ++nu) v0[nu] = gaussian_component(seed, vec_offset + (uint64_t)r, (uint64_t)nu);
    normalise(v0);
  } else if (start_mode == 3) {
    const uint64_t v = vec_offset + (uint64_t)r;
    std::vector<cplx> rk(M.dim);
    for (int64_t nu = 0; nu < M.dim; ++nu) rk[nu] = gaussian_component(seed, v / 2, (uint64_t)nu);
    normalise(rk);
    if (v % 2) time_reverse(M, rk.data(), v0.data(), 1);
    else v0 = rk;
  } else if (start_mode == 1) {
    const int64_t b = basis_offset + r;
    if (b < 0 || b >= M.dim) return false;
    v0[b] = 1.0;
  } else {
    const cplx* us = reinterpret_cast<const cplx*>(user_start);
    for (int64_t nu = 0; nu < M.dim; ++nu) v0[nu] = us[nu * R + r];
    normalise(v0);
  }
  return true;
}

}  // namespace

extern "C" {

int64_t oracle_dim(const oracle_system* s) {
  Model M;
  if (!build_model(s, M)) return -1;
  return M.dim;
}

// Pair tensor A_ij (3x3, row-major) as assembled from Eq. (3); for tests.
int oracle_pair_tensor(const oracle_system* s, int i, int j, double* out9) {
  Model M;
  if (!build_model(s, M) || i < 0 || j <= i || j >= M.n) return -1;
  std::memcpy(out9, &M.A[((size_t)i * M.n + j) * 9], 9 * sizeof(double));
  return 0;
}

// y = H x; x, y: [dim][nvec] complex (interleaved re, im).
int oracle_apply_h(const oracle_system* s, const double* x, double* y, int64_t nvec) {
  Model M;
  if (!build_model(s, M) || nvec <= 0) return -1;
  auto PL = all_pair_ladders(M);
  apply_h(M, PL, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y), nvec);
  return 0;
}

// y = (dir . S) x, S = sum_i s_i.
int oracle_apply_sdir(const oracle_system* s, const double* dir, const double* x, double* y,
                      int64_t nvec) {
  Model M;
  if (!build_model(s, M) || nvec <= 0) return -1;
  apply_sdir(M, dir, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y), nvec);
  return 0;
}

// y = Theta x (time reversal, Sec. II.B); x, y: [dim][nvec], not aliased.
int oracle_time_reverse(const oracle_system* s, const double* x, double* y, int64_t nvec) {
  Model M;
  if (!build_model(s, M) || nvec <= 0 || x == y) return -1;
  time_reverse(M, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y), nvec);
  return 0;
}

// Column nu of H, duplicates summed: rows[k], vals[2k], vals[2k+1].  Returns
// the number of entries, or -1.  cap bounds the output.
int64_t oracle_h_column(const oracle_system* s, int64_t nu, int64_t* rows, double* vals, int64_t cap) {
  Model M;
  if (!build_model(s, M) || nu < 0 || nu >= M.dim) return -1;
  auto PL = all_pair_ladders(M);
  std::vector<Entry> col;
  column_entries(M, PL, nu, col);
  std::sort(col.begin(), col.end(), [](const Entry& a, const Entry& b) { return a.row < b.row; });
  int64_t k = 0;
  for (size_t e = 0; e < col.size(); ++e) {
    if (k > 0 && rows[k - 1] == col[e].row) {
      vals[2 * (k - 1)] += col[e].val.real();
      vals[2 * (k - 1) + 1] += col[e].val.imag();
      continue;
    }
    if (k >= cap) return -1;
    rows[k] = col[e].row;
    vals[2 * k] = col[e].val.real();
    vals[2 * k + 1] = col[e].val.imag();
    ++k;
  }
  return k;
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox(ctr, key, out); }

// Start block [d][R]: column k is random vector number vec_offset + k,
// Gaussian components, normalised to 1.
int oracle_start_vectors(int64_t d, int64_t R, uint64_t seed, uint64_t vec_offset, double* out) {
  if (d <= 0 || R <= 0) return -1;
  cplx* o = reinterpret_cast<cplx*>(out);
  for (int64_t k = 0; k < R; ++k) {
    double nrm = 0.0;
    for (int64_t nu = 0; nu < d; ++nu) {
      cplx z = gaussian_component(seed, vec_offset + (uint64_t)k, (uint64_t)nu);
      o[nu * R + k] = z;
      nrm += std::norm(z);
    }
    nrm = std::sqrt(nrm);
    for (int64_t nu = 0; nu < d; ++nu) o[nu * R + k] /= nrm;
  }
  return 0;
}

// One Lanczos run from v0 (normalised inside).  Returns M_eff or -1.
int oracle_lanczos(const oracle_system* s, const double* v0, int maxM, int reorth, double tol,
                   const double* dir, double* alpha, double* beta, double* p) {
  Model M;
  if (!build_model(s, M) || maxM <= 0) return -1;
  auto PL = all_pair_ladders(M);
  std::vector<cplx> v(reinterpret_cast<const cplx*>(v0), reinterpret_cast<const cplx*>(v0) + M.dim);
  double nrm = 0.0;
  for (auto& z : v) nrm += std::norm(z);
  nrm = std::sqrt(nrm);
  if (!(nrm > 0.0)) return -1;
  for (auto& z : v) z /= nrm;
  const double* u = dir ? dir : M.Bdir;
  return lanczos(M, PL, v, maxM, reorth, tol, u, alpha, beta, reinterpret_cast<cplx*>(p));
}

int oracle_tridiag_eig(int m, const double* alpha, const double* beta, double* evals, double* evecs) {
  if (m <= 0) return -1;
  jacobi_tridiag(m, alpha, beta, evals, evecs);
  return 0;
}

// Eqs. (4), (5): thermodynamics from the tridiagonal data of R runs.
// alpha, beta: [R][M]; p: [R][M] complex; M_eff: [R].  Outputs per T: lnZ,
// E, C (k_B = 1), M_B = -g Re<dir.S>, M_B_imag = -g Im<dir.S>.  E0 = lowest
// Ritz value over all runs.
int oracle_ftlm_sums(int R, int maxM, const int* M_eff, const double* alpha, const double* beta,
                     const double* p, double dim, double g, const double* T, int nT, double* lnZ,
                     double* E, double* C, double* MB, double* MB_imag, double* E0_out) {
  if (R <= 0 || maxM <= 0 || nT <= 0) return -1;
  std::vector<std::vector<double>> ev(R), u0(R);
  std::vector<std::vector<cplx>> q(R);
  for (int r = 0; r < R; ++r)
    if (M_eff[r] <= 0 || M_eff[r] > maxM) return -1;
  // the R eigenproblems are independent: one host thread each (no shared writes)
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    const int m = M_eff[r];
    std::vector<double> U((size_t)m * m);
    ev[r].resize(m);
    jacobi_tridiag(m, alpha + (size_t)r * maxM, beta + (size_t)r * maxM, ev[r].data(), U.data());
    u0[r].resize(m);
    q[r].assign(m, 0.0);
    const cplx* pr = reinterpret_cast<const cplx*>(p) + (size_t)r * maxM;
    for (int nn = 0; nn < m; ++nn) {
      u0[r][nn] = U[nn];  // U_{0n}
      cplx acc = 0.0;
      for (int j = 0; j < m; ++j) acc += U[(size_t)j * m + nn] * std::conj(pr[j]);  // <r|O|n>
      q[r][nn] = acc;
    }
  }
  double E0 = INFINITY;
  for (int r = 0; r < R; ++r)
    for (double e : ev[r]) E0 = std::min(E0, e);
  for (int t = 0; t < nT; ++t) {
    const double b = 1.0 / T[t];
    double z = 0.0, e1 = 0.0;
    cplx o = 0.0;
    for (int r = 0; r < R; ++r)
      for (size_t nn = 0; nn < ev[r].size(); ++nn) {
        const double bz = std::exp(-b * (ev[r][nn] - E0));
        const double w = u0[r][nn] * u0[r][nn] * bz;
        z += w;
        e1 += w * ev[r][nn];
        o += bz * u0[r][nn] * q[r][nn];
      }
    const double Em = e1 / z;
    double var = 0.0;
    for (int r = 0; r < R; ++r)
      for (size_t nn = 0; nn < ev[r].size(); ++nn) {
        const double w = u0[r][nn] * u0[r][nn] * std::exp(-b * (ev[r][nn] - E0));
        var += w * (ev[r][nn] - Em) * (ev[r][nn] - Em);
      }
    lnZ[t] = std::log(dim / R * z) - b * E0;
    E[t] = Em;
    C[t] = b * b * var / z;
    MB[t] = -g * std::real(o) / z;
    MB_imag[t] = -g * std::imag(o) / z;
  }
  if (E0_out) *E0_out = E0;
  return 0;
}

// Full FTLM.  start_mode: 0 = Philox random vectors (vec_offset + k),
// 1 = basis vectors |basis_offset + k>, 2 = user block [d][R] (normalised per
// column inside).  alpha, beta, p, M_eff: outputs [R][M] (may be NULL).
// The Lanczos half of FTLM on its own: the R recurrences (one host thread
// each), returning their tridiagonal data alpha, beta, p [R][M] and M_eff [R].
int oracle_ftlm_tridiag(const oracle_system* s, int R, int maxM, uint64_t seed, uint64_t vec_offset,
                        int start_mode, int64_t basis_offset, const double* user_start, int reorth, double tol,
                        const double* dir, double* alpha_out, double* beta_out, double* p_out, int* meff_out) {
  Model M;
  if (!build_model(s, M) || R <= 0 || maxM <= 0) return -1;
  auto PL = all_pair_ladders(M);
  const double* u = dir ? dir : M.Bdir;
  std::vector<double> alpha((size_t)R * maxM, 0.0), beta((size_t)R * maxM, 0.0);
  std::vector<cplx> p((size_t)R * maxM, 0.0);
  std::vector<int> meff(R, 0);
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    std::vector<cplx> v0(M.dim, 0.0);
    if (!start_vector(M, r, R, seed, vec_offset, start_mode, basis_offset, user_start, v0)) {
#pragma omp atomic write
      fail = 1;
      continue;
    }
    meff[r] = lanczos(M, PL, v0, maxM, reorth, tol, u, &alpha[(size_t)r * maxM], &beta[(size_t)r * maxM],
                      &p[(size_t)r * maxM]);
  }
  if (fail) return -1;
  std::memcpy(alpha_out, alpha.data(), sizeof(double) * alpha.size());
  std::memcpy(beta_out, beta.data(), sizeof(double) * beta.size());
  std::memcpy(p_out, p.data(), sizeof(cplx) * p.size());
  std::memcpy(meff_out, meff.data(), sizeof(int) * meff.size());
  return 0;
}

int oracle_ftlm(const oracle_system* s, int R, int maxM, uint64_t seed, uint64_t vec_offset, int start_mode,
                int64_t basis_offset, const double* user_start, int reorth, double tol, const double* dir,
                const double* T, int nT, double* lnZ, double* E, double* C, double* MB, double* MB_imag,
                double* E0, double* alpha_out, double* beta_out, double* p_out, int* meff_out) {
  Model M;
  if (!build_model(s, M) || R <= 0 || maxM <= 0 || nT <= 0) return -1;
  std::vector<double> alpha((size_t)R * maxM, 0.0), beta((size_t)R * maxM, 0.0);
  std::vector<cplx> p((size_t)R * maxM, 0.0);
  std::vector<int> meff(R, 0);
  if (oracle_ftlm_tridiag(s, R, maxM, seed, vec_offset, start_mode, basis_offset, user_start, reorth, tol, dir,
                          alpha.data(), beta.data(), reinterpret_cast<double*>(p.data()), meff.data()) != 0)
    return -1;
  int rc = oracle_ftlm_sums(R, maxM, meff.data(), alpha.data(), beta.data(), reinterpret_cast<double*>(p.data()),
                            (double)M.dim, M.g, T, nT, lnZ, E, C, MB, MB_imag, E0);
  if (alpha_out) std::memcpy(alpha_out, alpha.data(), sizeof(double) * alpha.size());
  if (beta_out) std::memcpy(beta_out, beta.data(), sizeof(double) * beta.size());
  if (p_out) std::memcpy(p_out, p.data(), sizeof(cplx) * p.size());
  if (meff_out) std::memcpy(meff_out, meff.data(), sizeof(int) * meff.size());
  return rc;
}

// Symmetric FTLM for O = dir.S, Eqs. (E-2-G) and (E-2-H): per run r
//   <r|e^{-beta H/2} O e^{-beta H/2}|r> ~ sum_{m,n} e^{-beta (eps_m + eps_n)/2}
//        <r|m> <m|O|n> <n|r>,   <m|O|n> = sum_{i,j} U_im O_ij U_jn,
// O_ij = <v_i|O|v_j> in the Lanczos basis, <r|n> = U_0n; the denominator
// <r|e^{-beta H}|r> = sum_n e^{-beta eps_n} |U_0n|^2.  Both shifted by E0 (the
// lowest Ritz value over all runs).  Omat: [R][M][M] complex, Omat[r][i][j] =
// O_ij.  Outputs MB_sym = -g Re(num / den), MB_sym_imag = -g Im(num / den).
int oracle_sftlm_sums(int R, int maxM, const int* M_eff, const double* alpha, const double* beta,
                      const double* Omat, double g, const double* T, int nT, double* MB_sym, double* MB_sym_imag) {
  if (R <= 0 || maxM <= 0 || nT <= 0) return -1;
  std::vector<std::vector<double>> ev(R), U(R);
  std::vector<std::vector<cplx>> Ot(R);  // <m|O|n>
  double E0 = INFINITY;
  for (int r = 0; r < R; ++r) {
    const int m = M_eff[r];
    if (m <= 0 || m > maxM) return -1;
    ev[r].resize(m);
    U[r].resize((size_t)m * m);
    jacobi_tridiag(m, alpha + (size_t)r * maxM, beta + (size_t)r * maxM, ev[r].data(), U[r].data());
    for (int nn = 0; nn < m; ++nn) E0 = std::min(E0, ev[r][nn]);
    const cplx* O = reinterpret_cast<const cplx*>(Omat) + (size_t)r * maxM * maxM;
    Ot[r].assign((size_t)m * m, 0.0);
    for (int mm = 0; mm < m; ++mm)
      for (int nn = 0; nn < m; ++nn) {
        cplx acc = 0.0;
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j) acc += U[r][(size_t)i * m + mm] * O[(size_t)i * maxM + j] * U[r][(size_t)j * m + nn];
        Ot[r][(size_t)mm * m + nn] = acc;
      }
  }
  for (int t = 0; t < nT; ++t) {
    const double b = 1.0 / T[t];
    double den = 0.0;
    cplx num = 0.0;
    for (int r = 0; r < R; ++r) {
      const int m = M_eff[r];
      for (int nn = 0; nn < m; ++nn) den += std::exp(-b * (ev[r][nn] - E0)) * U[r][nn] * U[r][nn];
      for (int mm = 0; mm < m; ++mm)
        for (int nn = 0; nn < m; ++nn)
          num += std::exp(-0.5 * b * (ev[r][mm] + ev[r][nn] - 2.0 * E0)) * U[r][mm] * Ot[r][(size_t)mm * m + nn] *
                 U[r][nn];
    }
    MB_sym[t] = -g * std::real(num) / den;
    MB_sym_imag[t] = -g * std::imag(num) / den;
  }
  return 0;
}

// Lanczos runs that also return O_ij = <v_i|dir.S|v_j> for each run
// (Omat [R][M][M] complex, zero outside M_eff), with the start modes of
// oracle_ftlm; then the FTLM outputs of oracle_ftlm_sums and the sFTLM
// M_B of oracle_sftlm_sums.
int oracle_sftlm(const oracle_system* s, int R, int maxM, uint64_t seed, uint64_t vec_offset, int start_mode,
                 int64_t basis_offset, const double* user_start, int reorth, double tol, const double* dir,
                 const double* T, int nT, double* lnZ, double* E, double* C, double* MB, double* MB_imag,
                 double* MB_sym, double* MB_sym_imag, double* E0, double* alpha_out, double* beta_out,
                 double* Omat_out, int* meff_out) {
  Model M;
  if (!build_model(s, M) || R <= 0 || maxM <= 0 || nT <= 0) return -1;
  auto PL = all_pair_ladders(M);
  const double* u = dir ? dir : M.Bdir;
  std::vector<double> alpha((size_t)R * maxM, 0.0), beta((size_t)R * maxM, 0.0);
  std::vector<cplx> p((size_t)R * maxM, 0.0), O((size_t)R * maxM * maxM, 0.0);
  std::vector<int> meff(R, 0);
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < R; ++r) {
    std::vector<cplx> v0;
    if (!start_vector(M, r, R, seed, vec_offset, start_mode, basis_offset, user_start, v0)) {
#pragma omp atomic write
      fail = 1;
      continue;
    }
    std::vector<std::vector<cplx>> V;
    meff[r] = lanczos(M, PL, v0, maxM, reorth, tol, u, &alpha[(size_t)r * maxM], &beta[(size_t)r * maxM],
                      &p[(size_t)r * maxM], &V);
    std::vector<cplx> w(M.dim);
    for (int j = 0; j < meff[r]; ++j) {
      apply_sdir(M, u, V[j].data(), w.data(), 1);
      for (int i = 0; i < meff[r]; ++i) O[((size_t)r * maxM + i) * maxM + j] = dot(V[i], w);
    }
  }
  if (fail) return -1;
  int rc = oracle_ftlm_sums(R, maxM, meff.data(), alpha.data(), beta.data(), reinterpret_cast<double*>(p.data()),
                            (double)M.dim, M.g, T, nT, lnZ, E, C, MB, MB_imag, E0);
  if (rc == 0)
    rc = oracle_sftlm_sums(R, maxM, meff.data(), alpha.data(), beta.data(), reinterpret_cast<double*>(O.data()), M.g,
                           T, nT, MB_sym, MB_sym_imag);
  if (alpha_out) std::memcpy(alpha_out, alpha.data(), sizeof(double) * alpha.size());
  if (beta_out) std::memcpy(beta_out, beta.data(), sizeof(double) * beta.size());
  if (Omat_out) std::memcpy(Omat_out, O.data(), sizeof(cplx) * O.size());
  if (meff_out) std::memcpy(meff_out, meff.data(), sizeof(int) * meff.size());
  return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
