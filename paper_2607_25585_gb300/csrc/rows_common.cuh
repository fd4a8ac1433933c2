// Shared pieces of the general row kernels (kernels.cu) and the stored-matrix
// builder (csr.cu): the per-CTA shared-memory staging of one system's tables
// and the enumeration of the matrix elements of one row of H (Eq. 3).
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ftlm_internal.h"

namespace ftlm {

// ---------------------------------------------------------------------------
// shared-memory staging of one instance's tables
// ---------------------------------------------------------------------------
struct SmemView {
  void* tab;
  long long* stride;
  int* q;
  unsigned char* dig;   // [max_n][blockDim]  the row's digits, one column per thread
  void* mcol;           // [max_n][blockDim]  the row's m values (real), one column per thread
  double* red;          // [blockDim][kNumPartials * V]
};

template <typename real>
__device__ SmemView carve(unsigned char* raw, const LaunchArgs& a, int V) {
  SmemView s;
  size_t off = 0;
  s.tab = raw;
  off += ((size_t)a.tab_reals * sizeof(real) + 15) & ~size_t(15);
  s.stride = reinterpret_cast<long long*>(raw + off);
  off += (size_t)a.max_n * 8;
  s.q = reinterpret_cast<int*>(raw + off);
  off += ((size_t)a.max_n * 4 + 15) & ~size_t(15);
  s.red = reinterpret_cast<double*>(raw + off);
  off += (size_t)blockDim.x * kNumPartials * V * 8;
  s.mcol = raw + off;
  off += ((size_t)a.max_n * blockDim.x * sizeof(real) + 15) & ~size_t(15);
  s.dig = raw + off;
  return s;
}

template <typename real>
__device__ void stage_instance(const InstDesc& d, const SmemView& s) {
  const real* src = reinterpret_cast<const real*>(d.tab);
  real* dst = reinterpret_cast<real*>(s.tab);
  for (int i = threadIdx.x; i < d.lay.total; i += blockDim.x) dst[i] = src[i];
  for (int i = threadIdx.x; i < d.n; i += blockDim.x) {
    s.stride[i] = d.stride[i];
    s.q[i] = d.q[i];
  }
}

// ---------------------------------------------------------------------------
// the terms of one row of H (Eq. 3), general mixed radix.  Row mu couples to
// every nu with <mu|H|nu> != 0: the diagonal, single-site +-1 and +-2 steps,
// and the four +-1/+-1 pair steps of every pair i < j.  The sink receives
// diag(<mu|H|mu>) first, then term(nu, Re, Im) for every off-diagonal element
// <mu|H|nu> in a fixed order: the gather (h_row) accumulates them against x,
// the stored-matrix builder counts or writes them.
// ---------------------------------------------------------------------------
// (re, im, re, im) from a 16-byte-aligned shared-memory table entry
template <typename real>
struct Quad {
  real a, b, c, d;
};
template <typename real>
__device__ __forceinline__ Quad<real> ld4(const real* p) {
  if (sizeof(real) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {(real)v.x, (real)v.y, (real)v.z, (real)v.w};
  }
  const double2 u = *reinterpret_cast<const double2*>(p), w = *(reinterpret_cast<const double2*>(p) + 1);
  return {(real)u.x, (real)u.y, (real)w.x, (real)w.y};
}

template <typename real, typename Sink>
__device__ __forceinline__ void row_terms(const SmemView& s, const TabLayout& L, int n, long long mu, bool idx32,
                                          Sink& sink) {
  const real* t = reinterpret_cast<const real*>(s.tab);
  const int qm = L.qmax;
  unsigned char* dg = s.dig + threadIdx.x;
  real* mc = reinterpret_cast<real*>(s.mcol) + threadIdx.x;
  const int bd = blockDim.x;
  // mixed-radix digits of mu (site 0 least significant) and their m values
  if (idx32) {
    unsigned rem = (unsigned)mu;
    for (int i = 0; i < n; ++i) {
      const unsigned qi = (unsigned)s.q[i];
      const unsigned nq = rem / qi;
      const int a_i = (int)(rem - nq * qi);
      dg[i * bd] = (unsigned char)a_i;
      mc[i * bd] = t[L.off_m + i * qm + a_i];
      rem = nq;
    }
  } else {
    unsigned long long rem = (unsigned long long)mu;
    for (int i = 0; i < n; ++i) {
      const unsigned long long qi = (unsigned long long)s.q[i];
      const unsigned long long nq = rem / qi;
      const int a_i = (int)(rem - nq * qi);
      dg[i * bd] = (unsigned char)a_i;
      mc[i * bd] = t[L.off_m + i * qm + a_i];
      rem = nq;
    }
  }
  // diagonal: sum_{i<j} zz m_i m_j + sum_i (h_z m_i + single-ion diagonal)
  real diag = 0;
  for (int i = 0; i < n; ++i) {
    const real mi = mc[i * bd];
    real zsum = t[L.off_hz + i];
    for (int j = i + 1; j < n; ++j) zsum = fma(t[L.off_zz + i * n + j], mc[j * bd], zsum);
    diag = fma(mi, zsum, diag);
    diag += t[L.off_iondiag + i * qm + dg[i * bd]];
  }
  sink.diag(diag);
  for (int i = 0; i < n; ++i) {
    const int a_i = dg[i * bd];
    const int qi = s.q[i];
    const long long si = s.stride[i];
    const Quad<real> ti = ld4(t + L.off_site4 + 4 * (i * qm + a_i));  // up, dn, m, single-ion diagonal
    const real up_i = ti.a, dn_i = ti.b, mi = ti.c;
    // coefficient of the s+_i-type single steps: h+_i + sum_j rho_ij m_j
    real fr = t[L.off_hp + 2 * i], fi = t[L.off_hp + 2 * i + 1];
    for (int j = 0; j < n; ++j) {
      const real mj = mc[j * bd];
      const typename Cx<real>::v2 rho = *reinterpret_cast<const typename Cx<real>::v2*>(t + L.off_rho + 2 * (i * n + j));
      fr = fma(rho.x, mj, fr);
      fi = fma(rho.y, mj, fi);
    }
    const real bzr = t[L.off_bz + 2 * i], bzi = t[L.off_bz + 2 * i + 1];
    if (a_i >= 1) {  // mu = s+_i nu: (F + bz (2m - 1)) <a|s+|a-1>
      const real w = (real)2 * mi - (real)1;
      sink.term(mu - si, (fr + bzr * w) * up_i, (fi + bzi * w) * up_i);
    }
    if (a_i + 1 < qi) {  // mu = s-_i nu: conj(F + bz (2m + 1)) <a|s-|a+1>
      const real w = (real)2 * mi + (real)1;
      sink.term(mu + si, (fr + bzr * w) * dn_i, -(fi + bzi * w) * dn_i);
    }
    if (a_i >= 2) {
      const real u2 = t[L.off_up2 + i * qm + a_i];
      sink.term(mu - 2 * si, t[L.off_bb + 2 * i] * u2, t[L.off_bb + 2 * i + 1] * u2);
    }
    if (a_i + 2 < qi) {
      const real d2 = t[L.off_dn2 + i * qm + a_i];
      sink.term(mu + 2 * si, t[L.off_bb + 2 * i] * d2, -t[L.off_bb + 2 * i + 1] * d2);
    }
    for (int j = i + 1; j < n; ++j) {
      const int a_j = dg[j * bd];
      const int qj = s.q[j];
      const long long sj = s.stride[j];
      const Quad<real> tj = ld4(t + L.off_site4 + 4 * (j * qm + a_j));
      const real up_j = tj.a, dn_j = tj.b;
      const Quad<real> cij = ld4(t + L.off_pair4 + 4 * (i * n + j));  // s+_i s-_j and s+_i s+_j
      const real pmr = cij.a, pmi = cij.b, ppr = cij.c, ppi = cij.d;
      const bool iu = a_i >= 1, id = a_i + 1 < qi, ju = a_j >= 1, jd = a_j + 1 < qj;
      if (iu && jd) {  // mu = s+_i s-_j nu
        const real e = up_i * dn_j;
        sink.term(mu - si + sj, pmr * e, pmi * e);
      }
      if (id && ju) {  // mu = s-_i s+_j nu
        const real e = dn_i * up_j;
        sink.term(mu + si - sj, pmr * e, -pmi * e);
      }
      if (iu && ju) {  // mu = s+_i s+_j nu
        const real e = up_i * up_j;
        sink.term(mu - si - sj, ppr * e, ppi * e);
      }
      if (id && jd) {  // mu = s-_i s-_j nu
        const real e = dn_i * dn_j;
        sink.term(mu + si + sj, ppr * e, -ppi * e);
      }
    }
  }
}

// The gather: acc = <mu|H|mu> x_mu + sum_nu <mu|H|nu> x_nu for V vectors.
template <typename real, int V>
struct GatherSink {
  const void* x;
  long long mu;
  int R, col;
  real *ar, *ai, *xr_own, *xi_own;
  __device__ __forceinline__ void diag(real dv) {
    VecIO<real, V>::ldg(x, mu * R + col, xr_own, xi_own);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ar[v] = dv * xr_own[v];
      ai[v] = dv * xi_own[v];
    }
  }
  __device__ __forceinline__ void term(long long nu, real cr, real ci) {
    gather_mac<real, V>(x, nu, R, col, cr, ci, ar, ai);
  }
};

}  // namespace ftlm
