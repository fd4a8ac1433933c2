// Full re-orthogonalisation of the Lanczos recurrence (Sec. II.C of arxiv
// 2607.25585: the optional step that keeps the new vector orthogonal to all
// previous ones of its chain).  After w = H v_j - alpha_j v_j - beta_j v_{j-1}
// has been formed, each pass removes w's components along the stored vectors
//   w <- w - sum_{k <= j} v_k <v_k|w>,  v_k = sigma_k q_k,
// and the run applies two passes (Gram-Schmidt twice).  The coefficients are
// summed in FP64 in a fixed order (one warp per (vector, k), a fixed shuffle
// tree), so the result is bitwise reproducible.
//
// Layout: the stored vectors are vector-major, Vs[k][r][mu] (vector r of step
// k contiguous); the working block w is row-major [d][R]; the scales sigma are
// [M + 1][R] and the coefficients G are [R][M] complex, all FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "ftlm_internal.h"

namespace ftlm {

namespace {

// G[r][k] = <q_k | w_r> for k = 0..j: one warp per (k, r).
template <typename real>
__global__ void __launch_bounds__(256) reorth_dot_kernel(const real* __restrict__ Vs, const real* __restrict__ w,
                                                         long long d, int R, int j, int M, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int r = blockIdx.y;
  if (k > j) return;  // whole warps leave together
  const real* q = Vs + 2 * ((size_t)k * R + r) * (size_t)d;
  double sr = 0.0, si = 0.0;
  for (long long mu = lane; mu < d; mu += 32) {
    const double qr = q[2 * mu], qi = q[2 * mu + 1];
    const double wr = w[2 * (mu * R + r)], wi = w[2 * (mu * R + r) + 1];
    sr += qr * wr + qi * wi;  // conj(q) w
    si += qr * wi - qi * wr;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    G[2 * ((size_t)r * M + k)] = sr;
    G[2 * ((size_t)r * M + k) + 1] = si;
  }
}

// w_r[mu] -= sum_{k <= j} sigma_k^2 G[r][k] q_k[mu]: one thread per (mu, r).
template <typename real>
__global__ void __launch_bounds__(256) reorth_axpy_kernel(const real* __restrict__ Vs, real* __restrict__ w,
                                                          long long d, int R, int j, int M,
                                                          const double* __restrict__ G,
                                                          const double* __restrict__ sigma) {
  const long long mu = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (mu >= d) return;
  double ar = 0.0, ai = 0.0;
  for (int k = 0; k <= j; ++k) {
    const double sg = sigma[(size_t)k * R + r];
    const double gr = G[2 * ((size_t)r * M + k)] * sg * sg, gi = G[2 * ((size_t)r * M + k) + 1] * sg * sg;
    const real* q = Vs + 2 * (((size_t)k * R + r) * (size_t)d + mu);
    const double qr = q[0], qi = q[1];
    ar += gr * qr - gi * qi;
    ai += gr * qi + gi * qr;
  }
  real* wp = w + 2 * (mu * R + r);
  wp[0] = (real)((double)wp[0] - ar);
  wp[1] = (real)((double)wp[1] - ai);
}

}  // namespace

int launch_reorth_pass(const void* Vs, void* w, long long dim, int R, int j, int M, double* G, const double* sigma,
                       int c64, void* stream) {
  if (R < 1 || R > 65535 || j < 0 || j >= M) return (int)cudaErrorInvalidValue;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const dim3 gd((unsigned)((j + 1 + 7) / 8), (unsigned)R);
  const dim3 ga((unsigned)((dim + 255) / 256), (unsigned)R);
  if (c64) {
    reorth_dot_kernel<float><<<gd, 256, 0, st>>>(static_cast<const float*>(Vs), static_cast<const float*>(w), dim, R,
                                                 j, M, G);
    reorth_axpy_kernel<float><<<ga, 256, 0, st>>>(static_cast<const float*>(Vs), static_cast<float*>(w), dim, R, j,
                                                  M, G, sigma);
  } else {
    reorth_dot_kernel<double><<<gd, 256, 0, st>>>(static_cast<const double*>(Vs), static_cast<const double*>(w), dim,
                                                  R, j, M, G);
    reorth_axpy_kernel<double><<<ga, 256, 0, st>>>(static_cast<const double*>(Vs), static_cast<double*>(w), dim, R,
                                                   j, M, G, sigma);
  }
  return (int)cudaGetLastError();
}

}  // namespace ftlm
