// Stored-matrix comparison path: H of Eq. (3) assembled once as a sparse
// matrix in compressed-row form and multiplied with vector blocks.  The paper
// stores its matrix stripes on the GPUs in coordinate form, grouped so that
// one thread handles all elements of a row (Sec. II.C, Table I); compressed
// rows are that grouping written as row pointers.  The matrix-free gather is
// the hot path; this path exists to measure what storing the matrix costs and
// gains on one GB300.
//
// Assembly runs the same row enumeration as the gather (row_terms): a count
// pass, a prefix sum of the counts (CUB), and a fill pass.  Within a row the
// diagonal comes first, then the off-diagonal elements in the gather's order;
// elements whose value is exactly zero are not stored.
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "ftlm_internal.h"
#include "rows_common.cuh"

namespace ftlm {

namespace {

template <typename real>
struct CountSink {
  int n = 0;
  __device__ __forceinline__ void diag(real) { ++n; }
  __device__ __forceinline__ void term(long long, real cr, real ci) {
    if (cr != (real)0 || ci != (real)0) ++n;
  }
};

template <typename real>
struct FillSink {
  long long pos;
  long long mu;
  int* col;
  real* val;  // interleaved (re, im)
  __device__ __forceinline__ void diag(real dv) {
    col[pos] = (int)mu;
    val[2 * pos] = dv;
    val[2 * pos + 1] = (real)0;
    ++pos;
  }
  __device__ __forceinline__ void term(long long nu, real cr, real ci) {
    if (cr == (real)0 && ci == (real)0) return;
    col[pos] = (int)nu;
    val[2 * pos] = cr;
    val[2 * pos + 1] = ci;
    ++pos;
  }
};

// FILL = false: counts[mu] = stored elements of row mu; true: write the row at rp[mu].
template <typename real, bool FILL>
__global__ void __launch_bounds__(256) csr_rows_kernel(const __grid_constant__ LaunchArgs a, int* counts,
                                                       const long long* rp, int* col, real* val) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmemView s = carve<real>(smem_raw, a, 1);
  const InstDesc& d = a.one;
  stage_instance<real>(d, s);
  __syncthreads();
  const bool idx32 = d.dim <= 0xffffffffll;
  for (long long mu = blockIdx.x * (long long)blockDim.x + threadIdx.x; mu < d.dim;
       mu += (long long)gridDim.x * blockDim.x) {
    if (FILL) {
      FillSink<real> f{rp[mu], mu, col, val};
      row_terms<real>(s, d.lay, d.n, mu, idx32, f);
    } else {
      CountSink<real> c;
      row_terms<real>(s, d.lay, d.n, mu, idx32, c);
      counts[mu] = c.n;
    }
  }
}

// y[mu][k] = sum_e val[e] x[col[e]][k] over row mu's elements; a thread owns one
// row and a chunk of V consecutive vectors (C = R / V chunks per row), so with
// R = 64 (complex64) a warp reads one row's elements once and whole 512-byte
// rows of x.
template <typename real, int V>
__global__ void __launch_bounds__(256) csr_spmm_kernel(long long dim, int R, int C, const long long* __restrict__ rp,
                                                       const int* __restrict__ col, const real* __restrict__ val,
                                                       const void* __restrict__ x, void* __restrict__ y) {
  const long long items = dim * C;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const long long mu = it / C;
    const int c0 = (int)(it - mu * C) * V;
    real ar[V], ai[V];
#pragma unroll
    for (int v = 0; v < V; ++v) ar[v] = ai[v] = 0;
    const long long e1 = __ldg(rp + mu + 1);
    for (long long e = __ldg(rp + mu); e < e1; ++e) {
      const int nu = __ldg(col + e);
      const real cr = __ldg(val + 2 * e), ci = __ldg(val + 2 * e + 1);
      gather_mac<real, V>(x, nu, R, c0, cr, ci, ar, ai);
    }
    VecIO<real, V>::st(y, mu * R + c0, ar, ai);
  }
}

}  // namespace

size_t csr_smem_bytes(const LaunchArgs& a, int c64) {
  // the row kernels' staging layout with V = 1 (no reduction space is used)
  return rows_smem_bytes(a, c64, 256);
}

int csr_prepare(size_t smem) {
  const void* ks[] = {(const void*)csr_rows_kernel<float, false>, (const void*)csr_rows_kernel<float, true>,
                      (const void*)csr_rows_kernel<double, false>, (const void*)csr_rows_kernel<double, true>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

int launch_csr_count(const LaunchArgs& a, int c64, size_t smem, int* counts, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<long long>((a.one.dim + 255) / 256, 152LL * 8);
  if (c64) csr_rows_kernel<float, false><<<grid, 256, smem, st>>>(a, counts, nullptr, nullptr, nullptr);
  else csr_rows_kernel<double, false><<<grid, 256, smem, st>>>(a, counts, nullptr, nullptr, nullptr);
  return (int)cudaGetLastError();
}

int launch_csr_fill(const LaunchArgs& a, int c64, size_t smem, const long long* rp, int* col, void* val,
                    void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<long long>((a.one.dim + 255) / 256, 152LL * 8);
  if (c64) csr_rows_kernel<float, true><<<grid, 256, smem, st>>>(a, nullptr, rp, col, (float*)val);
  else csr_rows_kernel<double, true><<<grid, 256, smem, st>>>(a, nullptr, rp, col, (double*)val);
  return (int)cudaGetLastError();
}

// rp[0] = 0, rp[mu + 1] = sum_{nu <= mu} counts[nu]
int csr_scan(const int* counts, long long* rp, long long dim, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(rp, 0, sizeof(long long), st);
  if (e != cudaSuccess) return (int)e;
  size_t tmp = 0;
  e = cub::DeviceScan::InclusiveSum(nullptr, tmp, counts, rp + 1, (int)dim, st);
  if (e != cudaSuccess) return (int)e;
  void* buf = nullptr;
  e = cudaMallocAsync(&buf, tmp, st);
  if (e != cudaSuccess) return (int)e;
  e = cub::DeviceScan::InclusiveSum(buf, tmp, counts, rp + 1, (int)dim, st);
  cudaFreeAsync(buf, st);
  return (int)e;
}

int launch_csr_spmm(long long dim, int R, const long long* rp, const int* col, const void* val, const void* x,
                    void* y, int c64, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int V = (c64 && R % 2 == 0) ? 2 : 1;
  const int C = R / V;
  const long long items = dim * C;
  const int grid = (int)std::min<long long>((items + 255) / 256, 152LL * 16);
  if (c64 && V == 2)
    csr_spmm_kernel<float, 2><<<grid, 256, 0, st>>>(dim, R, C, rp, col, (const float*)val, x, y);
  else if (c64)
    csr_spmm_kernel<float, 1><<<grid, 256, 0, st>>>(dim, R, C, rp, col, (const float*)val, x, y);
  else
    csr_spmm_kernel<double, 1><<<grid, 256, 0, st>>>(dim, R, C, rp, col, (const double*)val, x, y);
  return (int)cudaGetLastError();
}

}  // namespace ftlm
