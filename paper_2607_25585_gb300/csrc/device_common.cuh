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

// V = 4, 8: complex64 values of V consecutive vectors, 16-byte loads
template <int V>
struct VecIOWide {
  static __device__ __forceinline__ void ldg(const void* b, long long idx, float* re, float* im) {
    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(b) + idx);
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
      const float4 t = __ldg(p + h);
      re[2 * h] = t.x; im[2 * h] = t.y; re[2 * h + 1] = t.z; im[2 * h + 1] = t.w;
    }
  }
  static __device__ __forceinline__ void ld(const void* b, long long idx, float* re, float* im) {
    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(b) + idx);
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
      const float4 t = p[h];
      re[2 * h] = t.x; im[2 * h] = t.y; re[2 * h + 1] = t.z; im[2 * h + 1] = t.w;
    }
  }
  static __device__ __forceinline__ void st(void* b, long long idx, const float* re, const float* im) {
    float4* p = reinterpret_cast<float4*>(reinterpret_cast<float2*>(b) + idx);
#pragma unroll
    for (int h = 0; h < V / 2; ++h) p[h] = make_float4(re[2 * h], im[2 * h], re[2 * h + 1], im[2 * h + 1]);
  }
};
template <>
struct VecIO<float, 4> : VecIOWide<4> {};
template <>
struct VecIO<float, 8> : VecIOWide<8> {};

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

// One element group of the elementwise modes: V consecutive values at
// complex index idx (V vectors of one row in the row-major block, or V rows of
// one vector in the vector-major block); sig, bsp, coef are their scalars:
//   Epilogue: sig = sigma_j, bsp = beta_{j-1} sigma_{j-1};
//   Step: the same and coef = alpha_j sigma_j;  Update: coef = alpha_j sigma_j;
//   Scale: coef = the factor.
// One element group of the recurrence step (kModeStep):
//   w = sigma H q_j - beta_j sigma_{j-1} q_{j-1} - alpha_j sigma_j q_j
// written over q_{j-1}, with the partials |w|^2 and <sigma q_j | u> (the p_j
// projection).  The loads are separate from the arithmetic and the store so
// that a thread can issue the loads of several groups before any store.
template <typename real, int V>
struct StepIn {
  real ar[V], ai[V], xr[V], xi[V], qr[V], qi[V], ur[V], ui[V];
};

template <typename real, int V>
__device__ __forceinline__ void step_load(const InstDesc& d, const LaunchArgs& a, long long idx, StepIn<real, V>& s) {
  VecIO<real, V>::ldg(d.hq, idx, s.ar, s.ai);
  for (int part = 1; part < a.hq_parts; ++part) {  // the passes' partial sums, in pass order
    real br[V], bi[V];
    VecIO<real, V>::ldg(d.hq, idx + part * a.hq_stride, br, bi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      s.ar[v] += br[v];
      s.ai[v] += bi[v];
    }
  }
  VecIO<real, V>::ldg(d.x, idx, s.xr, s.xi);
  VecIO<real, V>::ldg(d.u, idx, s.ur, s.ui);
  if (!a.first) {
    VecIO<real, V>::ld(d.y, idx, s.qr, s.qi);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) s.qr[v] = s.qi[v] = 0;
  }
}

template <typename real, int V>
__device__ __forceinline__ void step_finish(const InstDesc& d, long long idx, const StepIn<real, V>& s, const real* sig,
                                            const real* bsp, const real* coef, real* pacc) {
  real wr[V], wi[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    wr[v] = fma(sig[v], s.ar[v], fma(-bsp[v], s.qr[v], -coef[v] * s.xr[v]));
    wi[v] = fma(sig[v], s.ai[v], fma(-bsp[v], s.qi[v], -coef[v] * s.xi[v]));
  }
  VecIO<real, V>::st(d.y, idx, wr, wi);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const real vr = sig[v] * s.xr[v], vi = sig[v] * s.xi[v];
    pacc[v * kNumPartials + 0] += wr[v] * wr[v] + wi[v] * wi[v];
    pacc[v * kNumPartials + 1] += vr * s.ur[v] + vi * s.ui[v];
    pacc[v * kNumPartials + 2] += vr * s.ui[v] - vi * s.ur[v];
  }
}

// kModeStep over the groups e, e + step, ... < e_end, U groups' loads in
// flight per thread before their stores; the partials are summed in the same
// group order as one group at a time.
template <typename real, int V, int U>
__device__ __forceinline__ void step_stream(const InstDesc& d, const LaunchArgs& a, long long e, long long e_end,
                                            long long step, const real* sig, const real* bsp, const real* coef,
                                            real* pacc) {
  for (; e + (U - 1) * step < e_end; e += U * step) {
    StepIn<real, V> in[U];
#pragma unroll
    for (int k = 0; k < U; ++k) step_load<real, V>(d, a, e + k * step, in[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) step_finish<real, V>(d, e + k * step, in[k], sig, bsp, coef, pacc);
  }
  for (; e < e_end; e += step) {
    StepIn<real, V> in;
    step_load<real, V>(d, a, e, in);
    step_finish<real, V>(d, e, in, sig, bsp, coef, pacc);
  }
}

// kModeUpdate over the groups e, e + step, ... < e_end with U groups' loads in
// flight per thread before their stores: w -= coef q_j in place, partial |w|^2
// (summed in the same group order as one group at a time).
template <typename real, int V, int U>
__device__ __forceinline__ void update_stream(const InstDesc& d, long long e, long long e_end, long long step,
                                              const real* coef, real* pacc) {
  for (; e + (U - 1) * step < e_end; e += U * step) {
    real wr[U][V], wi[U][V], xr[U][V], xi[U][V];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      VecIO<real, V>::ld(d.y, e + k * step, wr[k], wi[k]);
      VecIO<real, V>::ldg(d.x, e + k * step, xr[k], xi[k]);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        wr[k][v] = fma(-coef[v], xr[k][v], wr[k][v]);
        wi[k][v] = fma(-coef[v], xi[k][v], wi[k][v]);
        pacc[v * kNumPartials] += wr[k][v] * wr[k][v] + wi[k][v] * wi[k][v];
      }
      VecIO<real, V>::st(d.y, e + k * step, wr[k], wi[k]);
    }
  }
  for (; e < e_end; e += step) {
    real wr[V], wi[V], xr[V], xi[V];
    VecIO<real, V>::ld(d.y, e, wr, wi);
    VecIO<real, V>::ldg(d.x, e, xr, xi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      wr[v] = fma(-coef[v], xr[v], wr[v]);
      wi[v] = fma(-coef[v], xi[v], wi[v]);
      pacc[v * kNumPartials] += wr[v] * wr[v] + wi[v] * wi[v];
    }
    VecIO<real, V>::st(d.y, e, wr, wi);
  }
}

// kModeEpilogue over the groups e, e + step, ... < e_end with U groups' loads
// in flight per thread before their stores: w = sigma H q_j - beta sigma' q_{j-1}
// in place of q_{j-1}, alpha and p partials (summed in the same group order
// as one group at a time).
template <typename real, int V, int U>
__device__ __forceinline__ void epilogue_stream(const InstDesc& d, const LaunchArgs& a, long long e, long long e_end,
                                                long long step, const real* sig, const real* bsp, real* pacc) {
  auto finish = [&](long long idx, const real* ar, const real* ai, const real* xr, const real* xi, const real* qr,
                    const real* qi, const real* ur, const real* ui) {
    real wr[V], wi[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      wr[v] = a.first ? sig[v] * ar[v] : fma(sig[v], ar[v], -bsp[v] * qr[v]);
      wi[v] = a.first ? sig[v] * ai[v] : fma(sig[v], ai[v], -bsp[v] * qi[v]);
    }
    VecIO<real, V>::st(d.y, idx, wr, wi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const real vr = sig[v] * xr[v], vi = sig[v] * xi[v];
      pacc[v * kNumPartials + 0] += vr * wr[v] + vi * wi[v];
      pacc[v * kNumPartials + 1] += vr * ur[v] + vi * ui[v];
      pacc[v * kNumPartials + 2] += vr * ui[v] - vi * ur[v];
    }
  };
  for (; e + (U - 1) * step < e_end; e += U * step) {
    real ar[U][V], ai[U][V], xr[U][V], xi[U][V], qr[U][V], qi[U][V], ur[U][V], ui[U][V];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      VecIO<real, V>::ldg(d.hq, e + k * step, ar[k], ai[k]);
      VecIO<real, V>::ldg(d.x, e + k * step, xr[k], xi[k]);
      VecIO<real, V>::ldg(d.u, e + k * step, ur[k], ui[k]);
      if (!a.first) {
        VecIO<real, V>::ld(d.y, e + k * step, qr[k], qi[k]);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) qr[k][v] = qi[k][v] = 0;
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) finish(e + k * step, ar[k], ai[k], xr[k], xi[k], qr[k], qi[k], ur[k], ui[k]);
  }
  for (; e < e_end; e += step) {
    real ar[V], ai[V], xr[V], xi[V], qr[V], qi[V], ur[V], ui[V];
    VecIO<real, V>::ldg(d.hq, e, ar, ai);
    VecIO<real, V>::ldg(d.x, e, xr, xi);
    VecIO<real, V>::ldg(d.u, e, ur, ui);
    if (!a.first) {
      VecIO<real, V>::ld(d.y, e, qr, qi);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) qr[v] = qi[v] = 0;
    }
    finish(e, ar, ai, xr, xi, qr, qi, ur, ui);
  }
}

template <typename real, int V, int MODE>
__device__ __forceinline__ void elementwise_item(const InstDesc& d, const LaunchArgs& a, long long idx,
                                                 const real* sig, const real* bsp, const real* coef, real* pacc) {
  if (MODE == kModeEpilogue) {  // w = sigma H q_j - beta sigma' q_{j-1}; alpha and p partials
    real ar[V], ai[V], xr[V], xi[V], wr[V], wi[V], ur[V], ui[V];
    VecIO<real, V>::ldg(d.hq, idx, ar, ai);
    VecIO<real, V>::ldg(d.x, idx, xr, xi);
    VecIO<real, V>::ldg(d.u, idx, ur, ui);
    if (!a.first) {
      real qr[V], qi[V];
      VecIO<real, V>::ld(d.y, idx, qr, qi);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        wr[v] = fma(sig[v], ar[v], -bsp[v] * qr[v]);
        wi[v] = fma(sig[v], ai[v], -bsp[v] * qi[v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        wr[v] = sig[v] * ar[v];
        wi[v] = sig[v] * ai[v];
      }
    }
    VecIO<real, V>::st(d.y, idx, wr, wi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const real vr = sig[v] * xr[v], vi = sig[v] * xi[v];
      pacc[v * kNumPartials + 0] += vr * wr[v] + vi * wi[v];
      pacc[v * kNumPartials + 1] += vr * ur[v] + vi * ui[v];
      pacc[v * kNumPartials + 2] += vr * ui[v] - vi * ur[v];
    }
  } else if (MODE == kModeStep) {  // w = sigma hq - bsp q_{j-1} - alpha sigma q_j; partials |w|^2, p
    StepIn<real, V> in;
    step_load<real, V>(d, a, idx, in);
    step_finish<real, V>(d, idx, in, sig, bsp, coef, pacc);
  } else if (MODE == kModeUpdate) {
    real wr[V], wi[V], xr[V], xi[V];
    VecIO<real, V>::ld(d.y, idx, wr, wi);
    VecIO<real, V>::ldg(d.x, idx, xr, xi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      wr[v] = fma(-coef[v], xr[v], wr[v]);
      wi[v] = fma(-coef[v], xi[v], wi[v]);
      pacc[v * kNumPartials] += wr[v] * wr[v] + wi[v] * wi[v];
    }
    VecIO<real, V>::st(d.y, idx, wr, wi);
  } else if (MODE == kModeStartNorm) {
    real xr[V], xi[V];
    VecIO<real, V>::ldg(d.x, idx, xr, xi);
#pragma unroll
    for (int v = 0; v < V; ++v) pacc[v * kNumPartials] += xr[v] * xr[v] + xi[v] * xi[v];
  } else if (MODE == kModeScale) {
    real xr[V], xi[V];
    VecIO<real, V>::ld(d.x, idx, xr, xi);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      xr[v] *= coef[v];
      xi[v] *= coef[v];
    }
    VecIO<real, V>::st(d.y, idx, xr, xi);
  }
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


// pair index of i < j in the triangular pair tables
__device__ __forceinline__ int tri(int i, int j) { return (j * (j - 1)) / 2 + i; }

// Complex accumulators.  FP32: two packed accumulators updated with the
// Blackwell f32x2 FMA, a = sum c_re x and b = sum c_im x (x = (re, im)), so a
// complex multiply-add is two FFMA2 and a real one (the s+ s- coefficients of
// a symmetric coupling tensor) is one; the value is (a.x - b.y, a.y + b.x).
// FP64: plain FMAs.
template <typename real>
struct Cx;

template <>
struct Cx<float> {
  using v2 = float2;
  float2 a, b;
  __device__ __forceinline__ void set(float e, float2 x) {
    a = make_float2(e * x.x, e * x.y);
    b = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void mac(float cr, float ci, float2 x) {
    a = __ffma2_rn(make_float2(cr, cr), x, a);
    b = __ffma2_rn(make_float2(ci, ci), x, b);
  }
  __device__ __forceinline__ void mac_re(float cr, float2 x) { a = __ffma2_rn(make_float2(cr, cr), x, a); }
  __device__ __forceinline__ void add(float2 v) {
    a.x += v.x;
    a.y += v.y;
  }
  __device__ __forceinline__ float2 value() const { return make_float2(a.x - b.y, a.y + b.x); }
};

template <>
struct Cx<double> {
  using v2 = double2;
  double re, im;
  __device__ __forceinline__ void set(double e, double2 x) {
    re = e * x.x;
    im = e * x.y;
  }
  __device__ __forceinline__ void mac(double cr, double ci, double2 x) {
    re = fma(cr, x.x, re);
    re = fma(-ci, x.y, re);
    im = fma(cr, x.y, im);
    im = fma(ci, x.x, im);
  }
  __device__ __forceinline__ void mac_re(double cr, double2 x) {
    re = fma(cr, x.x, re);
    im = fma(cr, x.y, im);
  }
  __device__ __forceinline__ void add(double2 v) {
    re += v.x;
    im += v.y;
  }
  __device__ __forceinline__ double2 value() const { return make_double2(re, im); }
};

template <typename real>
__device__ __forceinline__ typename Cx<real>::v2 ldx(const void* x, long long idx) {
  return __ldg(reinterpret_cast<const typename Cx<real>::v2*>(x) + idx);
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
      sc.alpha[(size_t)j * sc.ss + r] = total_partial(a, inst, r, 0);
      sc.p[((size_t)j * sc.ss + r) * 2] = total_partial(a, inst, r, 1);
      sc.p[((size_t)j * sc.ss + r) * 2 + 1] = total_partial(a, inst, r, 2);
    } else if (a.mode == kModeApply && a.fused_step) {  // alpha_j = Re<v_j|w'>, p_j = <v_j|u>
      const double sg = sc.sigma[(size_t)j * sc.ss + r];
      sc.alpha[(size_t)j * sc.ss + r] = sg * total_partial(a, inst, r, 0);
      sc.p[((size_t)j * sc.ss + r) * 2] = sg * total_partial(a, inst, r, 1);
      sc.p[((size_t)j * sc.ss + r) * 2 + 1] = sg * total_partial(a, inst, r, 2);
    } else if (a.mode == kModeApply) {  // gather_alpha
      const double sg = sc.sigma[(size_t)j * sc.ss + r];
      sc.alpha[(size_t)j * sc.ss + r] = sg * sg * total_partial(a, inst, r, 0);
    } else if (a.mode == kModeUpdate || a.mode == kModeStep) {
      if (a.mode == kModeStep) {
        sc.p[((size_t)j * sc.ss + r) * 2] = total_partial(a, inst, r, 1);
        sc.p[((size_t)j * sc.ss + r) * 2 + 1] = total_partial(a, inst, r, 2);
      }
      const double nrm2 = total_partial(a, inst, r, 0);
      const double bnew = sqrt(fmax(nrm2, 0.0));
      const double al = sc.alpha[(size_t)j * sc.ss + r];
      const double bold = j > 0 ? sc.beta[(size_t)(j - 1) * sc.ss + r] : 0.0;
      double scl = fmax(sc.scale[r], fmax(fabs(al), bold));
      sc.scale[r] = scl;
      sc.beta[(size_t)j * sc.ss + r] = bnew;
      double sig = 0.0;
      if (sc.active[r]) {
        if (j < d.M - 1 && (!(bnew > d.tol * scl) || !isfinite(bnew) || !isfinite(al))) {
          sc.active[r] = 0;
          sc.meff[r] = j + 1;
        } else {
          sig = bnew > 0.0 ? 1.0 / bnew : 0.0;
        }
      }
      sc.sigma[(size_t)(j + 1) * sc.ss + r] = sig;
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
