// General H.v (Eq. 3 of arxiv 2607.25585, any spins) on vector-major blocks
// with a register cube along the top site.
//
// Rows.  With T = n - 1 the top site (the largest stride s_T = dim / q_T), a
// row is mu = b + a s_T with b < s_T its "base" (the digits of sites 0..T-1)
// and a its top digit.  A thread owns one base b and all q_T = Q rows
// b + a s_T, for V vectors of one system (vector v at x + v dim); a warp's
// lanes own 32 consecutive bases, so every load is 32 consecutive values of
// one vector.
//
// Terms.  The digits, coefficients and validity of every term that does not
// involve the top site depend on b alone: they are formed once per base and
// applied to the Q x V values.  The top site's own flips (s+-_T, s+-2_T) move
// between rows of the cube (registers).  A flip of a lower site i loads the
// neighbouring cube x[b -+ s_i + a' s_T]: it serves the single flip of i (same
// a') and the pairs (i, T) (a' = a -+ 1), so the pairs with the top site cost
// no loads of their own.  The diagonal's top-site part, m_T(a) (h_T^z +
// sum_i zz_iT m_i) plus the single-ion diagonal of T, and the top-site part
// rho_iT m_T(a) of the single-flip coefficient of site i, are per row a.
//
// Terms follow the same coefficient conventions as the general row
// enumeration (rows_common.cuh); they are added in a different order, so
// results agree with it to rounding.
//
// Lanczos steps (a.fused_step): x = q_j, y = q_{j-1}, u; the epilogue writes
// w' = sigma_j H q_j - beta_j sigma_{j-1} q_{j-1} over q_{j-1} and sums
// Re<q_j|w'>, <q_j|u> per vector, so the step's update pass follows directly
// (no H q block and no separate epilogue pass); the last CTA sets alpha_j and
// p_j.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "ftlm_internal.h"
#include "rows_common.cuh"

namespace ftlm {

namespace {

template <typename real, int Q, int V>
__device__ __forceinline__ void load_cube(const typename Cx<real>::v2* x, long long dim, long long sT, long long nu,
                                          typename Cx<real>::v2 (&out)[Q][V]) {
#pragma unroll
  for (int a = 0; a < Q; ++a)
#pragma unroll
    for (int v = 0; v < V; ++v) out[a][v] = __ldg(x + (long long)v * dim + nu + (long long)a * sT);
}

// acc[a] += (cr + i ci) y for the V vectors of row a
template <typename real, int V>
__device__ __forceinline__ void cmac(real (&ar)[V], real (&ai)[V], real cr, real ci,
                                     const typename Cx<real>::v2 (&y)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    ar[v] = fma(cr, y[v].x, fma(-ci, y[v].y, ar[v]));
    ai[v] = fma(cr, y[v].y, fma(ci, y[v].x, ai[v]));
  }
}

template <typename real, int Q, int V>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? (Q * V <= 12 ? 3 : 2) : 1) cube_gather_kernel(const __grid_constant__ LaunchArgs a) {
  using v2 = typename Cx<real>::v2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmemView s = carve<real>(smem_raw, a, 0);
  __shared__ InstDesc d;
  // Lanczos step (a.fused_step): each thread's sums of Re<q_j|w'>, Re<q_j|u>,
  // Im<q_j|u> for the group's V vectors ([V * 3][256], a thread's own column),
  // the group's sigma_j and beta_j sigma_{j-1}, and the last CTA's flag
  __shared__ real sacc[V * 3 * 256];
  __shared__ double s_sg[V], s_bsp[V];
  __shared__ int is_last;
  const bool fused = a.fused_step != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const InstDesc* insts = a.inline_one ? &a.one : a.inst;
  const int nvec = a.n_inst * V;  // one-vector instances: the partial sums' slots [vector][CTA][kNumPartials]
  if (fused) {
    for (int k = threadIdx.x; k < nvec * kNumPartials; k += blockDim.x)
      a.partials[((size_t)(k / kNumPartials) * gridDim.x + blockIdx.x) * kNumPartials + k % kNumPartials] = 0.0;
    for (int k = threadIdx.x; k < V * 3 * 256; k += blockDim.x) sacc[k] = 0;
  }
  // the CTA's sums of group g's vectors into its partial slots: warp w adds
  // items w, w + 8, ... (item = vector x 3 + sum), lanes in a fixed order
  auto flush = [&](int g) {
    __syncthreads();
    for (int item = warp; item < V * 3; item += (int)(blockDim.x >> 5)) {
      double t = 0.0;
      for (int k = lane; k < (int)blockDim.x; k += 32) {
        t += (double)sacc[item * 256 + k];
        sacc[item * 256 + k] = 0;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0)
        a.partials[((size_t)(g * V + item / 3) * gridDim.x + blockIdx.x) * kNumPartials + item % 3] = t;
    }
    __syncthreads();
  };
  int cur = -1;
  const void* staged = nullptr;  // tables of the system now in shared memory
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int g = a.inline_one ? 0 : find_instance(a.tile_start, a.n_inst, tile);
    if (g != cur) {
      if (fused && cur >= 0) flush(cur);
      __syncthreads();
      if (threadIdx.x == 0) d = insts[(size_t)g * V];
      if (fused && threadIdx.x < V) {  // the group's vectors' step scalars
        const DevScalars& sc = insts[(size_t)g * V + threadIdx.x].sc;
        const int j = a.step;
        s_sg[threadIdx.x] = sc.sigma[(size_t)j * sc.ss];
        s_bsp[threadIdx.x] = a.first ? 0.0 : sc.beta[(size_t)(j - 1) * sc.ss] * sc.sigma[(size_t)(j - 1) * sc.ss];
      }
      __syncthreads();
      if (d.tab != staged) {  // the groups of one system share its tables
        stage_instance<real>(d, s);
        staged = d.tab;
      }
      cur = g;
      __syncthreads();
    }
    const int n = d.n, T = n - 1;
    const TabLayout& L = d.lay;
    const int qm = L.qmax;
    const real* t = reinterpret_cast<const real*>(s.tab);
    const long long dim = d.dim;
    const long long sT = s.stride[T];  // = dim / Q: the number of bases
    const int first_tile = a.inline_one ? 0 : __ldg(a.tile_start + g);
    const long long b0 = (long long)(tile - first_tile) * a.rows_per_tile;
    const long long b_end = min(b0 + a.rows_per_tile, sT);
    const v2* x = reinterpret_cast<const v2*>(d.x);
    v2* y = reinterpret_cast<v2*>(d.y);
    unsigned char* dg = s.dig + threadIdx.x;
    real* mc = reinterpret_cast<real*>(s.mcol) + threadIdx.x;
    const int bd = blockDim.x;
    // the top site's per-row tables: m, <a|s+|a-1>, <a|s-|a+1>, single-ion diagonal
    real mT[Q], upT[Q], dnT[Q], idT[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const Quad<real> tq = ld4(t + L.off_site4 + 4 * (T * qm + q));
      upT[q] = tq.a;
      dnT[q] = tq.b;
      mT[q] = tq.c;
      idT[q] = tq.d;
    }
    for (long long b = b0 + threadIdx.x; b < b_end; b += bd) {
      // digits of the base over sites 0..T-1 (its top digit is 0) and their m values
      {
        unsigned long long rem = (unsigned long long)b;
        unsigned rem32 = (unsigned)b;
        const bool idx32 = dim <= 0xffffffffll;
        for (int i = 0; i < T; ++i) {
          const unsigned qi = (unsigned)s.q[i];
          int ai;
          if (idx32) {
            const unsigned nq = rem32 / qi;
            ai = (int)(rem32 - nq * qi);
            rem32 = nq;
          } else {
            const unsigned long long nq = rem / qi;
            ai = (int)(rem - nq * qi);
            rem = nq;
          }
          dg[i * bd] = (unsigned char)ai;
          mc[i * bd] = t[L.off_m + i * qm + ai];
        }
      }
      // diagonal: the lower sites' part, and zT = sum_i zz_iT m_i; the top
      // site's single-flip coefficient F_T = h+_T + sum_i rho_Ti m_i
      real diag = 0, zT = 0;
      real fTr = t[L.off_hp + 2 * T], fTi = t[L.off_hp + 2 * T + 1];
      for (int i = 0; i < T; ++i) {
        const real mi = mc[i * bd];
        real zsum = t[L.off_hz + i];
        for (int j = i + 1; j < T; ++j) zsum = fma(t[L.off_zz + i * n + j], mc[j * bd], zsum);
        diag = fma(mi, zsum, diag);
        diag += t[L.off_iondiag + i * qm + dg[i * bd]];
        zT = fma(t[L.off_zz + i * n + T], mi, zT);
        fTr = fma(t[L.off_rho + 2 * (T * n + i)], mi, fTr);
        fTi = fma(t[L.off_rho + 2 * (T * n + i) + 1], mi, fTi);
      }
      real ar[Q][V], ai[Q][V];
      {
        v2 xo[Q][V];
        load_cube<real, Q, V>(x, dim, sT, b, xo);
        const real hzT = t[L.off_hz + T];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const real e = diag + mT[q] * (hzT + zT) + idT[q];
#pragma unroll
          for (int v = 0; v < V; ++v) {
            ar[q][v] = e * xo[q][v].x;
            ai[q][v] = e * xo[q][v].y;
          }
        }
        // the top site's flips, between rows of the cube
        const real bzr = t[L.off_bz + 2 * T], bzi = t[L.off_bz + 2 * T + 1];
        const real bbr = t[L.off_bb + 2 * T], bbi = t[L.off_bb + 2 * T + 1];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (q >= 1) {  // mu = s+_T nu: (F_T + bz (2m - 1)) <q|s+|q-1>
            const real w = (real)2 * mT[q] - (real)1;
            cmac<real, V>(ar[q], ai[q], (fTr + bzr * w) * upT[q], (fTi + bzi * w) * upT[q], xo[q - 1]);
          }
          if (q + 1 < Q) {  // mu = s-_T nu: conj(F_T + bz (2m + 1)) <q|s-|q+1>
            const real w = (real)2 * mT[q] + (real)1;
            cmac<real, V>(ar[q], ai[q], (fTr + bzr * w) * dnT[q], -(fTi + bzi * w) * dnT[q], xo[q + 1]);
          }
          if (q >= 2) {  // s+_T s+_T
            const real u2 = t[L.off_up2 + T * qm + q];
            cmac<real, V>(ar[q], ai[q], bbr * u2, bbi * u2, xo[q - 2]);
          }
          if (q + 2 < Q) {  // s-_T s-_T
            const real d2 = t[L.off_dn2 + T * qm + q];
            cmac<real, V>(ar[q], ai[q], bbr * d2, -bbi * d2, xo[q + 2]);
          }
        }
      }
      // the lower sites: single and double flips, pairs with the top site, pairs among themselves
      for (int i = 0; i < T; ++i) {
        const int a_i = dg[i * bd];
        const int qi = s.q[i];
        const long long si = s.stride[i];
        const Quad<real> ti = ld4(t + L.off_site4 + 4 * (i * qm + a_i));
        const real up_i = ti.a, dn_i = ti.b, mi = ti.c;
        real fr = t[L.off_hp + 2 * i], fi = t[L.off_hp + 2 * i + 1];
        for (int j = 0; j < T; ++j) {
          const real mj = mc[j * bd];
          const v2 rho = *reinterpret_cast<const v2*>(t + L.off_rho + 2 * (i * n + j));
          fr = fma(rho.x, mj, fr);
          fi = fma(rho.y, mj, fi);
        }
        const v2 rhoT = *reinterpret_cast<const v2*>(t + L.off_rho + 2 * (i * n + T));  // times m_T(row)
        const real bzr = t[L.off_bz + 2 * i], bzi = t[L.off_bz + 2 * i + 1];
        const Quad<real> cT = ld4(t + L.off_pair4 + 4 * (i * n + T));  // s+_i s-_T and s+_i s+_T
        if (a_i >= 1) {  // the cube at b - s_i
          v2 nb[Q][V];
          load_cube<real, Q, V>(x, dim, sT, b - si, nb);
          const real w = (real)2 * mi - (real)1;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            // mu = s+_i nu: (F_i + rho_iT m_T + bz (2m - 1)) <a_i|s+|a_i-1>
            cmac<real, V>(ar[q], ai[q], (fr + rhoT.x * mT[q] + bzr * w) * up_i, (fi + rhoT.y * mT[q] + bzi * w) * up_i,
                          nb[q]);
            if (q + 1 < Q) {  // mu = s+_i s-_T nu
              const real e = up_i * dnT[q];
              cmac<real, V>(ar[q], ai[q], cT.a * e, cT.b * e, nb[q + 1]);
            }
            if (q >= 1) {  // mu = s+_i s+_T nu
              const real e = up_i * upT[q];
              cmac<real, V>(ar[q], ai[q], cT.c * e, cT.d * e, nb[q - 1]);
            }
          }
        }
        if (a_i + 1 < qi) {  // the cube at b + s_i
          v2 nb[Q][V];
          load_cube<real, Q, V>(x, dim, sT, b + si, nb);
          const real w = (real)2 * mi + (real)1;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            // mu = s-_i nu: conj(F_i + rho_iT m_T + bz (2m + 1)) <a_i|s-|a_i+1>
            cmac<real, V>(ar[q], ai[q], (fr + rhoT.x * mT[q] + bzr * w) * dn_i, -(fi + rhoT.y * mT[q] + bzi * w) * dn_i,
                          nb[q]);
            if (q >= 1) {  // mu = s-_i s+_T nu
              const real e = dn_i * upT[q];
              cmac<real, V>(ar[q], ai[q], cT.a * e, -cT.b * e, nb[q - 1]);
            }
            if (q + 1 < Q) {  // mu = s-_i s-_T nu
              const real e = dn_i * dnT[q];
              cmac<real, V>(ar[q], ai[q], cT.c * e, -cT.d * e, nb[q + 1]);
            }
          }
        }
        if (a_i >= 2) {  // s+_i s+_i
          const real u2 = t[L.off_up2 + i * qm + a_i];
          const real cr = t[L.off_bb + 2 * i] * u2, ci = t[L.off_bb + 2 * i + 1] * u2;
          v2 nb[Q][V];
          load_cube<real, Q, V>(x, dim, sT, b - 2 * si, nb);
#pragma unroll
          for (int q = 0; q < Q; ++q) cmac<real, V>(ar[q], ai[q], cr, ci, nb[q]);
        }
        if (a_i + 2 < qi) {  // s-_i s-_i
          const real d2 = t[L.off_dn2 + i * qm + a_i];
          const real cr = t[L.off_bb + 2 * i] * d2, ci = -t[L.off_bb + 2 * i + 1] * d2;
          v2 nb[Q][V];
          load_cube<real, Q, V>(x, dim, sT, b + 2 * si, nb);
#pragma unroll
          for (int q = 0; q < Q; ++q) cmac<real, V>(ar[q], ai[q], cr, ci, nb[q]);
        }
        for (int j = i + 1; j < T; ++j) {  // pairs of two lower sites: one coefficient for the cube
          const int a_j = dg[j * bd];
          const int qj = s.q[j];
          const long long sj = s.stride[j];
          const Quad<real> tj = ld4(t + L.off_site4 + 4 * (j * qm + a_j));
          const Quad<real> cij = ld4(t + L.off_pair4 + 4 * (i * n + j));  // s+_i s-_j and s+_i s+_j
          const bool iu = a_i >= 1, id = a_i + 1 < qi, ju = a_j >= 1, jd = a_j + 1 < qj;
          auto pair = [&](long long nu, real cr, real ci) {
            v2 nb[Q][V];
            load_cube<real, Q, V>(x, dim, sT, nu, nb);
#pragma unroll
            for (int q = 0; q < Q; ++q) cmac<real, V>(ar[q], ai[q], cr, ci, nb[q]);
          };
          if (iu && jd) {  // mu = s+_i s-_j nu
            const real e = up_i * tj.b;
            pair(b - si + sj, cij.a * e, cij.b * e);
          }
          if (id && ju) {  // mu = s-_i s+_j nu
            const real e = dn_i * tj.a;
            pair(b + si - sj, cij.a * e, -cij.b * e);
          }
          if (iu && ju) {  // mu = s+_i s+_j nu
            const real e = up_i * tj.a;
            pair(b - si - sj, cij.c * e, cij.d * e);
          }
          if (id && jd) {  // mu = s-_i s-_j nu
            const real e = dn_i * tj.b;
            pair(b + si + sj, cij.c * e, -cij.d * e);
          }
        }
      }
      if (fused) {  // w' = sigma_j H q_j - beta_j sigma_{j-1} q_{j-1} over q_{j-1}; <q_j|w'>, <q_j|u>
        const v2* u = reinterpret_cast<const v2*>(d.u);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const real sg = (real)s_sg[v], bsp = (real)s_bsp[v];
          real pw = 0, pr = 0, pi = 0;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const long long e = (long long)v * dim + b + (long long)q * sT;
            v2 w;
            if (a.first) {
              w.x = sg * ar[q][v];
              w.y = sg * ai[q][v];
            } else {
              const v2 qp = __ldcs(y + e);
              w.x = sg * ar[q][v] - bsp * qp.x;
              w.y = sg * ai[q][v] - bsp * qp.y;
            }
            __stcs(y + e, w);
            const v2 xv = __ldg(x + e);  // own rows of q_j, re-read
            const v2 uv = __ldcs(u + e);
            pw += xv.x * w.x + xv.y * w.y;
            pr += xv.x * uv.x + xv.y * uv.y;
            pi += xv.x * uv.y - xv.y * uv.x;
          }
          sacc[(v * 3 + 0) * 256 + threadIdx.x] += pw;
          sacc[(v * 3 + 1) * 256 + threadIdx.x] += pr;
          sacc[(v * 3 + 2) * 256 + threadIdx.x] += pi;
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            v2 o;
            o.x = ar[q][v];
            o.y = ai[q][v];
            y[(long long)v * dim + b + (long long)q * sT] = o;
          }
      }
    }
  }
  if (!fused) return;
  // the last CTA to arrive sets alpha_j and p_j of every vector
  if (cur >= 0) flush(cur);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  LaunchArgs f = a;  // the vectors as one-vector instances
  f.n_inst = nvec;
  f.R = 1;
  f.mode = kModeApply;
  finalize(f, insts);
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <typename real, int Q, int V>
const void* cube_fn() {
  return (const void*)cube_gather_kernel<real, Q, V>;
}

// complex64: V = 8 or 4 vectors for cubes of 2 or 3 rows, 4 for 4..6 rows;
// complex128: 4 and 2
const void* cube_pick(int Q, int V, int c64) {
  if (c64) {
    if (Q == 2 && V == 8) return cube_fn<float, 2, 8>();
    if (Q == 2 && V == 4) return cube_fn<float, 2, 4>();
    if (Q == 3 && V == 8) return cube_fn<float, 3, 8>();
    if (Q == 3 && V == 4) return cube_fn<float, 3, 4>();
    if (Q == 4 && V == 4) return cube_fn<float, 4, 4>();
    if (Q == 5 && V == 4) return cube_fn<float, 5, 4>();
    if (Q == 6 && V == 4) return cube_fn<float, 6, 4>();
  } else {
    if (Q == 2 && V == 4) return cube_fn<double, 2, 4>();
    if (Q == 3 && V == 4) return cube_fn<double, 3, 4>();
    if (Q == 4 && V == 2) return cube_fn<double, 4, 2>();
    if (Q == 5 && V == 2) return cube_fn<double, 5, 2>();
    if (Q == 6 && V == 2) return cube_fn<double, 6, 2>();
  }
  return nullptr;
}

}  // namespace

int cube_vectors(int Q, int c64, int want) {
  if (want > 0) return cube_pick(Q, want, c64) ? want : 0;
  if (Q < 2 || Q > 6) return 0;
  return c64 ? (Q <= 3 ? 8 : 4) : (Q <= 3 ? 4 : 2);
}

int prepare_cube(int Q, int V, int c64, size_t smem) {
  const void* k = cube_pick(Q, V, c64);
  if (!k) return (int)cudaErrorInvalidValue;
  return (int)cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int cube_ctas_per_sm(int Q, int V, int c64, int threads, size_t smem) {
  const void* k = cube_pick(Q, V, c64);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess || n < 1) return 1;
  return n;
}

int launch_cube(const LaunchArgs& a, int Q, int V, int c64, int grid, int threads, size_t smem, void* stream) {
  const void* k = cube_pick(Q, V, c64);
  // (the step's per-thread sums are laid out for 256-thread CTAs)
  if (!k || a.mode != kModeApply || threads != 256) return (int)cudaErrorInvalidValue;
  void* args[] = {const_cast<LaunchArgs*>(&a)};
  return (int)cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace ftlm
