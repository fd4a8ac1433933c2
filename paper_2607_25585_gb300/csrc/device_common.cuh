// Device helpers shared by the row kernels: vector I/O of V complex values,
// the complex multiply-add, and the tile -> instance lookup.
#pragma once

#include <cuda_runtime.h>

#include "ftlm_internal.h"

namespace ftlm {

// ---------------------------------------------------------------------------
// vector I/O: V complex values of type real at complex index idx
// ---------------------------------------------------------------------------
template <typename real, int V>
struct VecIO;

template <>
struct VecIO<float, 2> {
  static __device__ __forceinline__ void ldg(const void* b, long long idx, float* re, float* im) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(b) + idx));
    re[0] = t.x; im[0] = t.y; re[1] = t.z; im[1] = t.w;
  }
  static __device__ __forceinline__ void ld(const void* b, long long idx, float* re, float* im) {
    const float4 t = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(b) + idx);
    re[0] = t.x; im[0] = t.y; re[1] = t.z; im[1] = t.w;
  }
  static __device__ __forceinline__ void st(void* b, long long idx, const float* re, const float* im) {
    *reinterpret_cast<float4*>(reinterpret_cast<float2*>(b) + idx) = make_float4(re[0], im[0], re[1], im[1]);
  }
};

template <>
struct VecIO<float, 1> {
  static __device__ __forceinline__ void ldg(const void* b, long long idx, float* re, float* im) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(b) + idx);
    re[0] = t.x; im[0] = t.y;
  }
  static __device__ __forceinline__ void ld(const void* b, long long idx, float* re, float* im) {
    const float2 t = reinterpret_cast<const float2*>(b)[idx];
    re[0] = t.x; im[0] = t.y;
  }
  static __device__ __forceinline__ void st(void* b, long long idx, const float* re, const float* im) {
    reinterpret_cast<float2*>(b)[idx] = make_float2(re[0], im[0]);
  }
};

template <>
struct VecIO<double, 1> {
  static __device__ __forceinline__ void ldg(const void* b, long long idx, double* re, double* im) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(b) + idx);
    re[0] = t.x; im[0] = t.y;
  }
  static __device__ __forceinline__ void ld(const void* b, long long idx, double* re, double* im) {
    const double2 t = reinterpret_cast<const double2*>(b)[idx];
    re[0] = t.x; im[0] = t.y;
  }
  static __device__ __forceinline__ void st(void* b, long long idx, const double* re, const double* im) {
    reinterpret_cast<double2*>(b)[idx] = make_double2(re[0], im[0]);
  }
};

// acc += c * x  for V complex values
template <typename real, int V>
__device__ __forceinline__ void cmac(real* ar, real* ai, real cr, real ci, const real* xr, const real* xi) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    ar[v] = fma(cr, xr[v], ar[v]);
    ar[v] = fma(-ci, xi[v], ar[v]);
    ai[v] = fma(cr, xi[v], ai[v]);
    ai[v] = fma(ci, xr[v], ai[v]);
  }
}

template <typename real, int V>
__device__ __forceinline__ void gather_mac(const void* x, long long nu, int R, int col, real cr, real ci, real* ar,
                                           real* ai) {
  real xr[V], xi[V];
  VecIO<real, V>::ldg(x, nu * R + col, xr, xi);
  cmac<real, V>(ar, ai, cr, ci, xr, xi);
}

__device__ __forceinline__ int find_instance(const int* tile_start, int n_inst, int tile) {
  if (n_inst == 1) return 0;
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile_start + mid) <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}


// Last CTA: total[inst][r][c] = sum over the CTAs' partials in a fixed order
// (four interleaved partial sums, combined in a fixed order), one thread per
// (inst, r, c): deterministic for a given grid.
__device__ inline double total_partial(const LaunchArgs& a, int inst, int r, int c) {
  const double* base = a.partials + (size_t)inst * gridDim.x * (size_t)a.R * kNumPartials + (size_t)r * kNumPartials + c;
  const size_t stride = (size_t)a.R * kNumPartials;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int b = 0;
  for (; b + 4 <= (int)gridDim.x; b += 4) {
    s0 += base[(size_t)b * stride];
    s1 += base[(size_t)(b + 1) * stride];
    s2 += base[(size_t)(b + 2) * stride];
    s3 += base[(size_t)(b + 3) * stride];
  }
  for (; b < (int)gridDim.x; ++b) s0 += base[(size_t)b * stride];
  return (s0 + s1) + (s2 + s3);
}

__device__ inline void finalize(const LaunchArgs& a, const InstDesc* inst_all) {
  // (inst_all points at the device array, or at the inline descriptor)
  const int R = a.R;
  for (int item = threadIdx.x; item < a.n_inst * R; item += blockDim.x) {
    const int inst = item / R, r = item % R;
    const InstDesc& d = inst_all[inst];
    const DevScalars& sc = d.sc;
    const int j = a.step;
    if (a.mode == kModeLanczos || a.mode == kModeEpilogue) {
      sc.alpha[(size_t)j * R + r] = total_partial(a, inst, r, 0);
      sc.p[((size_t)j * R + r) * 2] = total_partial(a, inst, r, 1);
      sc.p[((size_t)j * R + r) * 2 + 1] = total_partial(a, inst, r, 2);
    } else if (a.mode == kModeUpdate) {
      const double nrm2 = total_partial(a, inst, r, 0);
      const double bnew = sqrt(fmax(nrm2, 0.0));
      const double al = sc.alpha[(size_t)j * R + r];
      const double bold = j > 0 ? sc.beta[(size_t)(j - 1) * R + r] : 0.0;
      double scl = fmax(sc.scale[r], fmax(fabs(al), bold));
      sc.scale[r] = scl;
      sc.beta[(size_t)j * R + r] = bnew;
      double sig = 0.0;
      if (sc.active[r]) {
        if (j < d.M - 1 && (!(bnew > d.tol * scl) || !isfinite(bnew) || !isfinite(al))) {
          sc.active[r] = 0;
          sc.meff[r] = j + 1;
        } else {
          sig = bnew > 0.0 ? 1.0 / bnew : 0.0;
        }
      }
      sc.sigma[(size_t)(j + 1) * R + r] = sig;
    } else if (a.mode == kModeStartNorm) {
      const double nrm = sqrt(fmax(total_partial(a, inst, r, 0), 0.0));
      sc.sigma[r] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      sc.scale[r] = 0.0;
      sc.active[r] = nrm > 0.0 ? 1 : 0;
      sc.meff[r] = nrm > 0.0 ? d.M : 0;
    }
  }
}

}  // namespace ftlm
