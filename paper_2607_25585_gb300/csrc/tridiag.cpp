// Host half of FTLM (Eqs. 4-5 of arxiv 2607.25585): the tridiagonal
// eigenproblem of every Lanczos run and the Boltzmann sums.
//
// The eigenproblem uses the implicit QL iteration with shifts for symmetric
// tridiagonal matrices (Bowdler, Martin, Reinsch and Wilkinson, Numer. Math.
// 11, 1968).  The sums need only two rows of the eigenvector matrix U:
// U_0n (the weight <n|r>) and sum_j conj(p_j) U_jn (= <r|O|n>), so instead of
// accumulating the whole of U the plane rotations are applied to those row
// vectors only: O(M^2) per run instead of O(M^3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

#include "ftlm_internal.h"

namespace ftlm {

namespace {

// sqrt(a^2 + b^2): the plain formula where the squares can neither overflow
// nor underflow, the library's careful hypot elsewhere
inline double norm2(double a, double b) {
  const double m = std::max(std::fabs(a), std::fabs(b));
  if (m < 1e150 && m > 1e-150) return std::sqrt(a * a + b * b);
  return std::hypot(a, b);
}

// fn(i) for i in [0, n) on up to hardware_concurrency host threads (the
// caller's thread works too); each i runs exactly once
template <typename Fn>
void parallel_for(int n, Fn&& fn) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nth = std::min(std::min(n, hw), 32);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int i; (i = next.fetch_add(1)) < n;) fn(i);
  };
  std::vector<std::thread> pool;
  for (int k = 1; k < nth; ++k) {
    try {
      pool.emplace_back(work);
    } catch (...) {
      break;  // fewer threads: the others take the remaining items
    }
  }
  work();
  for (auto& t : pool) t.join();
}

// Eigenvalues of tridiag(d, e) (d[0..m-1], e[0..m-2] off-diagonal) with the
// rotations applied to the rows z[k][0..m-1], k < nz.  Returns false if the
// iteration does not converge.
bool ql_implicit(int m, double* d, double* e_in, int nz, double** z) {
  std::vector<double> e(m, 0.0);
  for (int i = 0; i + 1 < m; ++i) e[i] = e_in[i];
  const double eps = std::numeric_limits<double>::epsilon();
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    while (true) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        const double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
        if (std::fabs(e[mm]) <= eps * dd) break;
      }
      if (mm == l) break;
      if (++iter > 100) return false;
      // shift from the leading 2x2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = norm2(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = mm - 1;
      bool deflated = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = norm2(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // underflow: split the matrix here
          d[i + 1] -= p;
          e[mm] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        for (int k = 0; k < nz; ++k) {
          const double zi = z[k][i], zi1 = z[k][i + 1];
          z[k][i + 1] = s * zi + c * zi1;
          z[k][i] = c * zi - s * zi1;
        }
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  return true;
}

}  // namespace

ftlm_status host_sums(int R, int M, const int* M_eff, const double* alpha, const double* beta, const double* p,
                      double dim, double g, const double* T, int nT, ftlm_result* res, std::string& msg) {
  if (R < 1 || M < 1 || !M_eff || !alpha || !beta || !p || !T || nT < 1 || !res || !(dim > 0)) {
    msg = "ftlm_sums: invalid arguments";
    return FTLM_ERR_INVALID_ARG;
  }
  for (int t = 0; t < nT; ++t)
    if (!(T[t] > 0.0) || !std::isfinite(T[t])) {
      msg = "temperatures must be positive and finite";
      return FTLM_ERR_INVALID_ARG;
    }
  struct Run {
    std::vector<double> eps, w0, qr, qi;  // Ritz values, U_0n, Re/Im of sum_j conj(p_j) U_jn
  };
  std::vector<Run> runs(R);
  for (int r = 0; r < R; ++r)
    if (M_eff[r] < 1 || M_eff[r] > M) {
      msg = "M_eff out of range";
      return FTLM_ERR_INVALID_ARG;
    }
  // the runs' eigenproblems are independent: one per host thread
  std::vector<int> bad(R, 0);  // 1: non-finite coefficient, 2: no convergence
  parallel_for(R, [&](int r) {
    const int m = M_eff[r];
    Run& run = runs[r];
    run.eps.assign(alpha + (size_t)r * M, alpha + (size_t)r * M + m);
    std::vector<double> e(m > 1 ? m - 1 : 1, 0.0);
    for (int j = 0; j + 1 < m; ++j) e[j] = beta[(size_t)r * M + j];
    run.w0.assign(m, 0.0);
    run.w0[0] = 1.0;
    run.qr.resize(m);
    run.qi.resize(m);
    for (int j = 0; j < m; ++j) {  // conj(p_j)
      run.qr[j] = p[((size_t)r * M + j) * 2];
      run.qi[j] = -p[((size_t)r * M + j) * 2 + 1];
    }
    for (int j = 0; j < m; ++j)
      if (!std::isfinite(run.eps[j]) || (j + 1 < m && !std::isfinite(e[j]))) {
        bad[r] = 1;
        return;
      }
    double* rows[3] = {run.w0.data(), run.qr.data(), run.qi.data()};
    if (!ql_implicit(m, run.eps.data(), e.data(), 3, rows)) bad[r] = 2;
  });
  double E0 = std::numeric_limits<double>::infinity();
  for (int r = 0; r < R; ++r) {
    if (bad[r] == 1) {
      msg = "non-finite Lanczos coefficient in run " + std::to_string(r);
      return FTLM_ERR_NUMERICAL;
    }
    if (bad[r] == 2) {
      msg = "tridiagonal eigensolver did not converge (run " + std::to_string(r) + ")";
      return FTLM_ERR_NUMERICAL;
    }
    for (double v : runs[r].eps) E0 = std::min(E0, v);
  }
  res->E0 = E0;
  // the temperatures are independent too (each sums the runs in order)
  parallel_for(nT, [&](int t) {
    const double b = 1.0 / T[t];
    double z = 0.0, e1 = 0.0, orr = 0.0, oi = 0.0;
    for (const Run& run : runs)
      for (size_t n = 0; n < run.eps.size(); ++n) {
        const double boltz = std::exp(-b * (run.eps[n] - E0));
        const double w = run.w0[n] * run.w0[n] * boltz;
        z += w;
        e1 += w * run.eps[n];
        orr += boltz * run.w0[n] * run.qr[n];
        oi += boltz * run.w0[n] * run.qi[n];
      }
    const double Em = e1 / z;
    double var = 0.0;
    for (const Run& run : runs)
      for (size_t n = 0; n < run.eps.size(); ++n) {
        const double w = run.w0[n] * run.w0[n] * std::exp(-b * (run.eps[n] - E0));
        var += w * (run.eps[n] - Em) * (run.eps[n] - Em);
      }
    if (res->lnZ) res->lnZ[t] = std::log(dim / R * z) - b * E0;
    if (res->E) res->E[t] = Em;
    if (res->C) res->C[t] = b * b * var / z;
    if (res->M_B) res->M_B[t] = -g * orr / z;
    if (res->M_B_imag) res->M_B_imag[t] = -g * oi / z;
  });
  return FTLM_OK;
}

// Symmetric FTLM for O = u.S, Eqs. (E-2-G), (E-2-H): per run,
//   num_r = sum_{m,n} e^{-beta (eps_m + eps_n)/2} U_0m <m|O|n> U_0n = y^T O y,
//   y_i = sum_n U_in e^{-beta eps_n / 2} U_0n,
// with O_ij = <v_i|O|v_j> in the Lanczos basis (<m|O|n> = (U^T O U)_mn, U real),
// den_r = sum_n e^{-beta eps_n} U_0n^2; both shifted by E0, the lowest Ritz value
// over all runs.  Omat[r][i][j] (complex, row-major, M x M per run).  The whole
// of U is accumulated here: O(M^3) per run.
ftlm_status host_sums_sym(int R, int M, const int* M_eff, const double* alpha, const double* beta,
                          const double* Omat, double g, const double* T, int nT, double* MB_sym, double* MB_sym_imag,
                          std::string& msg) {
  if (R < 1 || M < 1 || !M_eff || !alpha || !beta || !Omat || !T || nT < 1) {
    msg = "sFTLM sums: invalid arguments";
    return FTLM_ERR_INVALID_ARG;
  }
  struct Run {
    int m = 0;
    std::vector<double> eps, U;  // U[k * m + n] = U_kn
  };
  std::vector<Run> runs(R);
  for (int r = 0; r < R; ++r)
    if (M_eff[r] < 1 || M_eff[r] > M) {
      msg = "M_eff out of range";
      return FTLM_ERR_INVALID_ARG;
    }
  std::vector<int> bad(R, 0);
  parallel_for(R, [&](int r) {
    Run& run = runs[r];
    const int m = run.m = M_eff[r];
    run.eps.assign(alpha + (size_t)r * M, alpha + (size_t)r * M + m);
    std::vector<double> e(m > 1 ? m - 1 : 1, 0.0);
    for (int j = 0; j + 1 < m; ++j) e[j] = beta[(size_t)r * M + j];
    run.U.assign((size_t)m * m, 0.0);
    std::vector<double*> rows(m);
    for (int k = 0; k < m; ++k) {
      run.U[(size_t)k * m + k] = 1.0;
      rows[k] = run.U.data() + (size_t)k * m;
    }
    if (!ql_implicit(m, run.eps.data(), e.data(), m, rows.data())) bad[r] = 1;
  });
  double E0 = std::numeric_limits<double>::infinity();
  for (int r = 0; r < R; ++r) {
    if (bad[r]) {
      msg = "tridiagonal eigensolver did not converge (run " + std::to_string(r) + ")";
      return FTLM_ERR_NUMERICAL;
    }
    for (double v : runs[r].eps) E0 = std::min(E0, v);
  }
  parallel_for(nT, [&](int t) {
    const double b = 1.0 / T[t];
    double den = 0.0, nre = 0.0, nim = 0.0;
    for (int r = 0; r < R; ++r) {
      const Run& run = runs[r];
      const int m = run.m;
      std::vector<double> x(m), y(m, 0.0);
      for (int n = 0; n < m; ++n) {
        const double h = std::exp(-0.5 * b * (run.eps[n] - E0));
        x[n] = h * run.U[n];  // U_0n
        den += h * h * run.U[n] * run.U[n];
      }
      for (int i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int n = 0; n < m; ++n) acc += run.U[(size_t)i * m + n] * x[n];
        y[i] = acc;
      }
      const double* O = Omat + (size_t)r * M * M * 2;
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          const double w = y[i] * y[j];
          nre += w * O[((size_t)i * M + j) * 2];
          nim += w * O[((size_t)i * M + j) * 2 + 1];
        }
    }
    MB_sym[t] = -g * nre / den;
    if (MB_sym_imag) MB_sym_imag[t] = -g * nim / den;
  });
  return FTLM_OK;
}

}  // namespace ftlm
