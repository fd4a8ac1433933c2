// The matrices of the observable in the Lanczos basis for the symmetric
// estimator (sFTLM, Eqs. E-2-G and E-2-H of arxiv 2607.25585): for every
// start vector r,
//   G_r[i][j] = <q_i | (u.S) q_j> = sum_mu conj(q_i[mu]) ((u.S) q_j)[mu],
// i, j < M, over the stored unnormalised Lanczos vectors q_k (O_ij =
// sigma_i sigma_j G_ij is formed on the host).  u.S = u_z S^z + a S^+ +
// conj(a) S^-, a = (u_x - i u_y)/2, is one-body, so (u.S) q_j at a row needs
// q_j at the row itself and at its single-site neighbours mu -+ stride_k.
//
// One kernel does both halves: a CTA owns one vector r, a 64 x 64 block of
// (i, j) and a range of rows.  Per tile of 32 rows (16 in complex128) it stages q_i (the i block)
// and (u.S) q_j (the j block, formed from the neighbours on the fly) in
// shared memory, and every thread accumulates 4 x 4 entries of G (rows
// ti + 16a, columns tj + 16b of the block) in registers.  (u.S) q_j is never
// written to device memory.  The CTA writes its partial block; a second
// kernel adds the partials of all row ranges in a fixed order in FP64
// (deterministic for a given launch shape).
//
// Stored vectors: vector-major, q_k of chain r at Vs + ((k R + r) dim) (k the
// Lanczos step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_common.cuh"

namespace ftlm {

namespace {

constexpr int kSymBlock = 64;  // i and j block
constexpr int kSymThreads = 256;

// rows per shared-memory tile: 32 complex64 or 16 complex128 (under 48 KB)
template <typename real>
struct SymRows {
  static constexpr int value = sizeof(real) == 4 ? 32 : 16;
};

template <typename real>
struct SymSmem {
  static constexpr int kRows = SymRows<real>::value;
  typename Cx<real>::v2 A[kSymBlock][kRows + 1];  // q_i[mu], i in the i block
  typename Cx<real>::v2 B[kSymBlock][kRows + 1];  // ((u.S) q_j)[mu], j in the j block
  real msum[kRows];                               // sum_k m_k(mu)
  unsigned char dig[kRows][kMaxSites];            // digits a_k(mu)
};

// grid: x = row range, y = (i block, j block), z = vector r.  Gp partials
// [r][range][M][M] complex FP64 (this CTA's block only).
template <typename real>
__global__ void __launch_bounds__(kSymThreads) sym_omat_kernel(const InstDesc d, const real* __restrict__ Vs, int R,
                                                             int M, long long rows_per_range, int nbj,
                                                             double* __restrict__ Gp) {
  using v2 = typename Cx<real>::v2;
  constexpr int kSymRows = SymRows<real>::value;
  __shared__ SymSmem<real> S;
  const int r = blockIdx.z;
  const int ib = blockIdx.y / nbj, jb = blockIdx.y % nbj;
  const int i0 = ib * kSymBlock, j0 = jb * kSymBlock;
  const int ni = min(kSymBlock, M - i0), nj = min(kSymBlock, M - j0);
  const long long dim = d.dim;
  const long long mu_lo = (long long)blockIdx.x * rows_per_range;
  const long long mu_hi = min(dim, mu_lo + rows_per_range);
  const real* t = reinterpret_cast<const real*>(d.tab);
  const TabLayout& L = d.lay;
  const int qm = L.qmax, n = d.n;
  const real uz = (real)d.obs[0], aur = (real)d.obs[1], aui = (real)d.obs[2];
  const size_t vstride = (size_t)R * (size_t)dim;  // elements between steps k and k + 1
  const v2* base = reinterpret_cast<const v2*>(Vs) + (size_t)r * (size_t)dim;
  // this thread's entries of the 64 x 64 block: rows ti + 16a, columns tj + 16b
  // (a half-warp reads 16 consecutive rows of B: no bank conflicts)
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  real gr[4][4], gi[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) gr[a][b] = gi[a][b] = 0;

  for (long long m0 = mu_lo; m0 < mu_hi; m0 += kSymRows) {
    const int nt = (int)min((long long)kSymRows, mu_hi - m0);
    __syncthreads();
    // digits and the S^z sum of the tile's rows
    for (int tt = threadIdx.x; tt < nt; tt += blockDim.x) {
      unsigned long long rem = (unsigned long long)(m0 + tt);
      real ms = 0;
      for (int k = 0; k < n; ++k) {
        const unsigned qk = (unsigned)__ldg(d.q + k);
        const unsigned long long nq = rem / qk;
        const int a = (int)(rem - nq * qk);
        rem = nq;
        S.dig[tt][k] = (unsigned char)a;
        ms += t[L.off_m + k * qm + a];
      }
      S.msum[tt] = ms;
    }
    // q_i of the i block
    for (int e = threadIdx.x; e < kSymBlock * kSymRows; e += blockDim.x) {
      const int ii = e / kSymRows, tt = e % kSymRows;
      v2 v;
      v.x = 0;
      v.y = 0;
      if (ii < ni && tt < nt) v = __ldg(base + (size_t)(i0 + ii) * vstride + (size_t)(m0 + tt));
      S.A[ii][tt] = v;
    }
    __syncthreads();
    // (u.S) q_j of the j block from the single-site neighbours
    for (int e = threadIdx.x; e < kSymBlock * kSymRows; e += blockDim.x) {
      const int jj = e / kSymRows, tt = e % kSymRows;
      v2 o;
      o.x = 0;
      o.y = 0;
      if (jj < nj && tt < nt) {
        const v2* x = base + (size_t)(j0 + jj) * vstride;
        const long long mu = m0 + tt;
        real ar = 0, ai = 0;
        for (int k = 0; k < n; ++k) {
          const int a = S.dig[tt][k];
          const int qk = __ldg(d.q + k);
          const long long st = __ldg(d.stride + k);
          if (a >= 1) {  // a S^+ : from mu - stride
            const real c = t[L.off_up1 + k * qm + a];
            const v2 xv = __ldg(x + mu - st);
            ar += c * (aur * xv.x - aui * xv.y);
            ai += c * (aur * xv.y + aui * xv.x);
          }
          if (a + 1 < qk) {  // conj(a) S^- : from mu + stride
            const real c = t[L.off_dn1 + k * qm + a];
            const v2 xv = __ldg(x + mu + st);
            ar += c * (aur * xv.x + aui * xv.y);
            ai += c * (aur * xv.y - aui * xv.x);
          }
        }
        const v2 xv = __ldg(x + mu);
        const real dz = uz * S.msum[tt];
        o.x = ar + dz * xv.x;
        o.y = ai + dz * xv.y;
      }
      S.B[jj][tt] = o;
    }
    __syncthreads();
    // G[i][j] += conj(A[i][mu]) B[j][mu]
    for (int tt = 0; tt < nt; ++tt) {
      v2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = S.A[ti + 16 * a][tt];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = S.B[tj + 16 * b][tt];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          gr[a][b] = fma(av[a].x, bv[b].x, fma(av[a].y, bv[b].y, gr[a][b]));
          gi[a][b] = fma(av[a].x, bv[b].y, fma(-av[a].y, bv[b].x, gi[a][b]));
        }
    }
  }
  // this CTA's partial block
  double* out = Gp + ((size_t)r * gridDim.x + blockIdx.x) * (size_t)M * M * 2;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * b;
      if (ti + 16 * a < ni && tj + 16 * b < nj) {
        out[2 * ((size_t)i * M + j)] = (double)gr[a][b];
        out[2 * ((size_t)i * M + j) + 1] = (double)gi[a][b];
      }
    }
}

// G[r][i][j] = sum over the row ranges of the partials, in range order.
__global__ void sym_reduce_kernel(const double* __restrict__ Gp, int R, int M, int nranges, double* __restrict__ G) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)M * M;
  if (e >= (long long)R * per) return;
  const long long r = e / per, ij = e % per;
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < nranges; ++k) {
    const double* p = Gp + ((size_t)(r * nranges + k) * per + ij) * 2;
    sr += p[0];
    si += p[1];
  }
  G[2 * e] = sr;
  G[2 * e + 1] = si;
}

}  // namespace

size_t sym_partial_doubles(int R, int M, int nranges) { return (size_t)R * nranges * M * M * 2; }

int sym_ranges(long long dim, int R, int M) {
  const int nb = (M + kSymBlock - 1) / kSymBlock;
  const long long blocks_per_range = (long long)R * nb * nb;
  // about four CTAs per SM in total, ranges of at least one tile and at most 2^13 rows
  long long ranges = std::max<long long>(1, (4LL * 152 + blocks_per_range - 1) / blocks_per_range);
  ranges = std::max<long long>(ranges, (dim + 8191) / 8192);
  ranges = std::min<long long>(ranges, (dim + 15) / 16);
  return (int)std::min<long long>(ranges, 1 << 20);
}

int launch_sym_omat(const InstDesc* h, const void* Vs, int R, int M, int nranges, double* Gp, double* G, int c64,
                    void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (R < 1 || R > 65535 || M < 1 || nranges < 1 || h->n > kMaxSites) return (int)cudaErrorInvalidValue;
  const int nb = (M + kSymBlock - 1) / kSymBlock;
  if ((long long)nb * nb > 65535) return (int)cudaErrorInvalidValue;
  const long long rows = (h->dim + nranges - 1) / nranges;
  const dim3 grid((unsigned)nranges, (unsigned)(nb * nb), (unsigned)R);
  if (c64) sym_omat_kernel<float><<<grid, kSymThreads, 0, st>>>(*h, (const float*)Vs, R, M, rows, nb, Gp);
  else sym_omat_kernel<double><<<grid, kSymThreads, 0, st>>>(*h, (const double*)Vs, R, M, rows, nb, Gp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  const long long total = (long long)R * M * M;
  sym_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Gp, R, M, nranges, G);
  return (int)cudaGetLastError();
}

}  // namespace ftlm
