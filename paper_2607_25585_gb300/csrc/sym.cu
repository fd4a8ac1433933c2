// The matrices of the observable in the Lanczos basis for the symmetric
// estimator (sFTLM, Eqs. E-2-G and E-2-H of arxiv 2607.25585): for every
// start vector r,
//   G_r[i][j] = <q_i | (u.S) q_j> = sum_mu conj(q_i[mu]) ((u.S) q_j)[mu],
// i, j < M, over the stored unnormalised Lanczos vectors q_k (O_ij =
// sigma_i sigma_j G_ij is formed on the host).  u.S = u_z S^z + a S^+ +
// conj(a) S^-, a = (u_x - i u_y)/2, is one-body, so (u.S) q_j at a row needs
// q_j at the row itself and at its single-site neighbours mu -+ stride_k.
//
// W_k = (u.S) q_k is formed first for every stored vector, vector after
// vector so that each vector's single-site neighbourhood stays in L2; then a
// contraction kernel in which a CTA owns one vector r, a 16T x 16T block of
// (i, j) and a range of rows.  Per tile of 64 rows (32 in complex128) it
// stages q_i (the i block) and W_j (the j block) in shared memory, and every
// thread accumulates T x T entries of G (rows ti + 16a, columns tj + 16b of
// the block) in registers.  The CTA writes its partial block; a second
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

constexpr int kSymBlock = 64;  // the largest i and j block (T = 4)
constexpr int kSymThreads = 256;

// rows per shared-memory tile: 64 complex64 or 32 complex128
template <typename real>
struct SymRows {
  static constexpr int value = sizeof(real) == 4 ? 64 : 32;
};

// Dynamic shared memory: the A and B tiles of blocks of 16 T vectors.
template <typename real, int T>
struct SymLayout {
  static constexpr int kRows = SymRows<real>::value;
  static constexpr int kPitch = kRows + 1;
  static constexpr int kB = 16 * T;
  static size_t tile_bytes() { return sizeof(typename Cx<real>::v2) * kB * kPitch; }
};

// The contraction G_r = Q_r^H W_r over blocks of kB = 16 T vectors (T x T
// entries a thread; T = 3 covers M = 40 with 48-blocks instead of padding it
// to 64).  grid: x = row range, y = (i block, j block), z = vector r.  Gp
// partials [r][range][M][M] complex FP64 (this CTA's block only).  The next
// tile's loads are issued into registers before the current tile's
// multiply-adds (all of a thread's loads in flight at once), so their latency
// is hidden behind the arithmetic instead of paid once per element.
template <typename real, int T>
__global__ void __launch_bounds__(kSymThreads, sizeof(real) == 4 ? 2 : 1) sym_omat_kernel(const real* __restrict__ Vs,
                                                               const real* __restrict__ Wv, long long dim, int R,
                                                               int M, long long rows_per_range, int nbj,
                                                               double* __restrict__ Gp) {
  using v2 = typename Cx<real>::v2;
  using Lay = SymLayout<real, T>;
  constexpr int kRows = Lay::kRows, kPitch = Lay::kPitch, kB = Lay::kB;
  constexpr int kPer = kB * kRows / kSymThreads;  // tile elements per thread
  static_assert(kB * kRows % kSymThreads == 0, "tile elements per thread");
  extern __shared__ __align__(16) unsigned char smem[];
  v2* A = reinterpret_cast<v2*>(smem);  // [kB][kPitch]
  v2* B = A + kB * kPitch;              // [kB][kPitch]
  const int r = blockIdx.z;
  const int ib = blockIdx.y / nbj, jb = blockIdx.y % nbj;
  const int i0 = ib * kB, j0 = jb * kB;
  const int ni = min(kB, M - i0), nj = min(kB, M - j0);
  const long long mu_lo = (long long)blockIdx.x * rows_per_range;
  const long long mu_hi = min(dim, mu_lo + rows_per_range);
  const size_t vstride = (size_t)R * (size_t)dim;
  const v2* abase = reinterpret_cast<const v2*>(Vs) + (size_t)r * (size_t)dim + (size_t)i0 * vstride;
  const v2* bbase = reinterpret_cast<const v2*>(Wv) + (size_t)r * (size_t)dim + (size_t)j0 * vstride;
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  const int na = (ni - ti + 15) / 16, nbb = (nj - tj + 15) / 16;
  real gr[T][T], gi[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) gr[a][b] = gi[a][b] = 0;
  v2 pa[kPer], pb[kPer];
  auto load = [&](long long m0) {
    const int nt = (int)min((long long)kRows, mu_hi - m0);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = threadIdx.x + u * kSymThreads;
      const int k = e / kRows, tt = e % kRows;
      pa[u].x = pa[u].y = pb[u].x = pb[u].y = 0;
      if (k < ni && tt < nt) pa[u] = __ldg(abase + (size_t)k * vstride + (size_t)(m0 + tt));
      if (k < nj && tt < nt) pb[u] = __ldg(bbase + (size_t)k * vstride + (size_t)(m0 + tt));
    }
  };
  if (mu_lo < mu_hi) load(mu_lo);
  for (long long m0 = mu_lo; m0 < mu_hi; m0 += kRows) {
    const int nt = (int)min((long long)kRows, mu_hi - m0);
    __syncthreads();  // the previous tile's multiply-adds are done
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = threadIdx.x + u * kSymThreads;
      const int k = e / kRows, tt = e % kRows;
      A[k * kPitch + tt] = pa[u];
      B[k * kPitch + tt] = pb[u];
    }
    __syncthreads();
    if (m0 + kRows < mu_hi) load(m0 + kRows);
    for (int tt = 0; tt < nt; ++tt) {
      v2 av[T], bv[T];
#pragma unroll
      for (int a = 0; a < T; ++a) av[a] = A[(ti + 16 * a) * kPitch + tt];
#pragma unroll
      for (int b = 0; b < T; ++b) bv[b] = B[(tj + 16 * b) * kPitch + tt];
#pragma unroll
      for (int a = 0; a < T; ++a) {
        if (a >= na) break;
#pragma unroll
        for (int b = 0; b < T; ++b) {
          if (b >= nbb) break;
          gr[a][b] = fma(av[a].x, bv[b].x, fma(av[a].y, bv[b].y, gr[a][b]));
          gi[a][b] = fma(av[a].x, bv[b].y, fma(-av[a].y, bv[b].x, gi[a][b]));
        }
      }
    }
  }
  double* out = Gp + ((size_t)r * gridDim.x + blockIdx.x) * (size_t)M * M * 2;
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int i = i0 + ti + 16 * a, j = j0 + tj + 16 * b;
      if (a < na && b < nbb) {
        out[2 * ((size_t)i * M + j)] = (double)gr[a][b];
        out[2 * ((size_t)i * M + j) + 1] = (double)gi[a][b];
      }
    }
}

// W_k = (u.S) q_k for every stored vector k (Vs order), V consecutive stored
// vectors a thread (the row's digits and coefficients formed once for them),
// row tiles of one group in consecutive CTAs (blockIdx.x fastest) so that the
// group's single-site neighbourhood is read from HBM once and then served by L2.
template <typename real, int V>
__global__ void __launch_bounds__(256) sym_sdir_kernel(const InstDesc d, const real* __restrict__ Vs,
                                                     real* __restrict__ Wv, int rows_per_cta) {
  using v2 = typename Cx<real>::v2;
  const real* t = reinterpret_cast<const real*>(d.tab);
  const TabLayout& L = d.lay;
  const int qm = L.qmax, n = d.n;
  const real uz = (real)d.obs[0], aur = (real)d.obs[1], aui = (real)d.obs[2];
  const long long dim = d.dim;
  const v2* x = reinterpret_cast<const v2*>(Vs) + (size_t)blockIdx.y * V * (size_t)dim;
  v2* w = reinterpret_cast<v2*>(Wv) + (size_t)blockIdx.y * V * (size_t)dim;
  const long long lo = (long long)blockIdx.x * rows_per_cta;
  const long long hi = min(dim, lo + rows_per_cta);
  const bool idx32 = dim <= 0xffffffffll;  // 32-bit digit division when the rows allow it
  for (long long mu = lo + threadIdx.x; mu < hi; mu += blockDim.x) {
    unsigned long long rem = (unsigned long long)mu;
    unsigned rem32 = (unsigned)mu;
    real ar[V], ai[V], ms = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) ar[v] = ai[v] = 0;
    for (int k = 0; k < n; ++k) {
      const int qk = __ldg(d.q + k);
      int a;
      if (idx32) {
        const unsigned nq = rem32 / (unsigned)qk;
        a = (int)(rem32 - nq * (unsigned)qk);
        rem32 = nq;
      } else {
        const unsigned long long nq = rem / (unsigned long long)qk;
        a = (int)(rem - nq * (unsigned long long)qk);
        rem = nq;
      }
      ms += t[L.off_m + k * qm + a];
      const long long st = __ldg(d.stride + k);
      if (a >= 1) {  // a S^+ : from mu - stride
        const real c = t[L.off_up1 + k * qm + a];
        const real cr = c * aur, ci = c * aui;
        v2 xv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) xv[v] = __ldg(x + (size_t)v * dim + mu - st);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          ar[v] += cr * xv[v].x - ci * xv[v].y;
          ai[v] += cr * xv[v].y + ci * xv[v].x;
        }
      }
      if (a + 1 < qk) {  // conj(a) S^- : from mu + stride
        const real c = t[L.off_dn1 + k * qm + a];
        const real cr = c * aur, ci = c * aui;
        v2 xv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) xv[v] = __ldg(x + (size_t)v * dim + mu + st);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          ar[v] += cr * xv[v].x + ci * xv[v].y;
          ai[v] += cr * xv[v].y - ci * xv[v].x;
        }
      }
    }
    const real dz = uz * ms;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const v2 xv = __ldg(x + (size_t)v * dim + mu);
      v2 o;
      o.x = ar[v] + dz * xv.x;
      o.y = ai[v] + dz * xv.y;
      w[(size_t)v * dim + mu] = o;
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

namespace {

template <typename real, int T>
cudaError_t launch_omat(const void* Vs, const void* W, long long dim, int R, int M, int nranges, double* Gp,
                        cudaStream_t st) {
  constexpr int kB = SymLayout<real, T>::kB;
  const int nb = (M + kB - 1) / kB;
  if ((long long)nb * nb > 65535) return cudaErrorInvalidValue;
  const long long rows = (dim + nranges - 1) / nranges;
  const dim3 grid((unsigned)nranges, (unsigned)(nb * nb), (unsigned)R);
  const size_t smem = 2 * SymLayout<real, T>::tile_bytes();
  cudaError_t e = cudaFuncSetAttribute(sym_omat_kernel<real, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sym_omat_kernel<real, T><<<grid, kSymThreads, smem, st>>>((const real*)Vs, (const real*)W, dim, R, M, rows, nb, Gp);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_omat_t(const void* Vs, const void* W, long long dim, int R, int M, int nranges, double* Gp,
                          cudaStream_t st) {
  const int T = std::min(4, (M + 15) / 16);  // the smallest blocks that cover M (at most 64)
  if (T == 1) return launch_omat<real, 1>(Vs, W, dim, R, M, nranges, Gp, st);
  if (T == 2) return launch_omat<real, 2>(Vs, W, dim, R, M, nranges, Gp, st);
  if (T == 3) return launch_omat<real, 3>(Vs, W, dim, R, M, nranges, Gp, st);
  return launch_omat<real, 4>(Vs, W, dim, R, M, nranges, Gp, st);
}

}  // namespace

int launch_sym_omat(const InstDesc* h, const void* Vs, void* W, int R, int M, int nranges, double* Gp, double* G,
                    int c64, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!W || R < 1 || R > 65535 || M < 1 || nranges < 1 || h->n > kMaxSites) return (int)cudaErrorInvalidValue;
  if ((long long)R * M > 65535) return (int)cudaErrorInvalidValue;
  const long long dim = h->dim;
  cudaError_t e;
  {  // (u.S) q_k of every stored vector, vector by vector
    const int trows = 1024;
    const int nv = R * M, V = nv % 8 == 0 ? 8 : (nv % 4 == 0 ? 4 : (nv % 2 == 0 ? 2 : 1));
    const dim3 g1((unsigned)((dim + trows - 1) / trows), (unsigned)(nv / V));
    if (c64) {
      if (V == 8) sym_sdir_kernel<float, 8><<<g1, 256, 0, st>>>(*h, (const float*)Vs, (float*)W, trows);
      else if (V == 4) sym_sdir_kernel<float, 4><<<g1, 256, 0, st>>>(*h, (const float*)Vs, (float*)W, trows);
      else if (V == 2) sym_sdir_kernel<float, 2><<<g1, 256, 0, st>>>(*h, (const float*)Vs, (float*)W, trows);
      else sym_sdir_kernel<float, 1><<<g1, 256, 0, st>>>(*h, (const float*)Vs, (float*)W, trows);
    } else {
      if (V == 8) sym_sdir_kernel<double, 8><<<g1, 256, 0, st>>>(*h, (const double*)Vs, (double*)W, trows);
      else if (V == 4) sym_sdir_kernel<double, 4><<<g1, 256, 0, st>>>(*h, (const double*)Vs, (double*)W, trows);
      else if (V == 2) sym_sdir_kernel<double, 2><<<g1, 256, 0, st>>>(*h, (const double*)Vs, (double*)W, trows);
      else sym_sdir_kernel<double, 1><<<g1, 256, 0, st>>>(*h, (const double*)Vs, (double*)W, trows);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
  }
  e = c64 ? launch_omat_t<float>(Vs, W, dim, R, M, nranges, Gp, st)
          : launch_omat_t<double>(Vs, W, dim, R, M, nranges, Gp, st);
  if (e != cudaSuccess) return (int)e;
  const long long total = (long long)R * M * M;
  sym_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Gp, R, M, nranges, G);
  return (int)cudaGetLastError();
}

}  // namespace ftlm
