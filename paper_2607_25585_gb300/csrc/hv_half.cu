// Spin-1/2 H.v (Eq. 3 of arxiv 2607.25585 with every s_i = 1/2): the
// matrix-free row gather specialised to the binary basis, where every pair
// (i, j) couples row mu to exactly one state mu ^ (e_i | e_j) and every site to
// mu ^ e_i.
//
// Register cubes.  A thread owns 2^K consecutive rows (the low K bits vary)
// of one vector.  Flips of the K cube bits stay in registers; a flip of an
// outer bit j loads the neighbouring cube once and serves the single flip of
// j and the K mixed pairs (c, j); an outer pair (i, j) has one coefficient for
// the whole cube.  This cuts the gathered loads per row from N(N+1)/2 to
// 1 + (N-K) + (N-K)(N-K-1)/2 and amortises coefficient work over 2^K rows.
//
// Coefficients.  Per system (once per CTA, in shared memory): the four
// coefficients of every pair indexed by the row's two bits, the cube part of
// the single-flip coefficients and of the diagonal.  Per row tile: the outer
// part of the single-flip coefficients and of the diagonal for every cube.
//
// Vector groups.  Vectors are processed Rg at a time (tile order is
// group-major), so the gathered slice x[:, group] (d * Rg * 8 bytes) stays in
// L2 while all its neighbours are read.
//
// Passes.  With one pass (cube on the low K bits) every pair of two outer
// bits costs one gathered load per multiply-add.  With ceil(N/K) passes
// whose cubes cover all N bits, every pair has an endpoint in some cube and
// is a mixed pair of that pass (K multiply-adds per gathered load); the
// gathered loads per row drop from 1 + (N-K) + C(N-K, 2) to about
// N/K + K C(N/K, 2), at the price of re-reading and re-writing the output in
// every pass after the first.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace ftlm {

namespace {

template <typename real>
struct HalfSmem {
  real* cp;     // [npairs][4][2]  coefficient by (bit_i, bit_j) of the row: 0=(0,0) 1=(0,1) 2=(1,0) 3=(1,1)
  real* fcube;  // [n][NR][2]      sum_{c<K} rho_jc m_c(r)
  real* ecube;  // [NR]            diagonal from the cube bits alone
  real* fhi;    // [n][Gt][2]      h+_j + sum_{i>=K} rho_ji m_i   per cube of the tile
  real* ehi;    // [Gt]            diagonal from the outer bits alone
  real* gz;     // [K][Gt]         sum_{i>=K} zz_ci m_i (cube-outer cross term)
  double* red;  // [blockDim][4]
};

template <typename real>
__device__ HalfSmem<real> half_carve(unsigned char* raw, int n, int K, int Gt) {
  HalfSmem<real> s;
  const int NR = 1 << K;
  const int npairs = n * (n - 1) / 2;
  real* p = reinterpret_cast<real*>(raw);
  s.cp = p;
  p += npairs * 8;
  s.fcube = p;
  p += n * NR * 2;
  s.ecube = p;
  p += NR;
  s.fhi = p;
  p += n * Gt * 2;
  s.ehi = p;
  p += Gt;
  s.gz = p;
  p += K * Gt;
  size_t off = (reinterpret_cast<unsigned char*>(p) - raw + 15) & ~size_t(15);
  s.red = reinterpret_cast<double*>(raw + off);
  return s;
}

}  // namespace

size_t half_smem_bytes(int n, int K, int rows_per_tile, int threads) {
  const int NR = 1 << K, Gt = rows_per_tile >> K;
  const size_t reals = (size_t)(n * (n - 1) / 2) * 8 + (size_t)n * NR * 2 + NR + (size_t)n * Gt * 2 + Gt + (size_t)K * Gt;
  // sized for double tables; float tables use less
  return ((reals * 8 + 15) & ~size_t(15)) + (size_t)threads * 4 * 8;
}

// RS > 0: the row stride R is the compile-time constant RS; RS = 0: runtime R.
// MP: one pass of the multi-pass form (cube position and pass flags from the
// launch arguments); otherwise the single-pass form with the cube on the low
// K bits, every choice known at compile time.
// MINB: resident CTAs per SM the register allocator must allow (2 or 3).
template <typename real, int K, int MODE, int RS, bool MP, int MINB>
__global__ void __launch_bounds__(256, MINB) half_kernel(const __grid_constant__ LaunchArgs a) {
  using v2 = typename Cx<real>::v2;
  constexpr int NR = 1 << K;
  // partial sums: alpha and p of the fused step, or Re<x|Hx> of a gather for the split step
  const bool kPartials = MODE == kModeLanczos || (MODE == kModeApply && !MP && a.gather_alpha);
  constexpr int NPS = MODE == kModeLanczos ? 3 : 1;  // partial sums in use
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDesc d;
  __shared__ int is_last;
  if (threadIdx.x == 0) d = a.inline_one ? a.one : a.inst[0];
  __syncthreads();
  const int n = d.n;
  const int Gt = a.rows_per_tile >> K;
  const HalfSmem<real> S = half_carve<real>(smem_raw, n, K, Gt);
  const real* t = reinterpret_cast<const real*>(d.tab);
  const TabLayout& L = d.lay;
  const int bd = blockDim.x;
  const int Rg = a.Rg;
  const int kl = threadIdx.x % Rg;
  const int slot = threadIdx.x / Rg, slots = bd / Rg;
  const int R = RS > 0 ? RS : a.R;
  const int s0 = MP ? a.cube_lo : 0;              // cube bits [s0, s0 + K)
  const int cnew = MP ? a.new_lo - s0 : 0;        // cube-relative first own bit
  const bool first = MP ? a.first_pass != 0 : true;
  const int later_lo = MP ? a.later_lo : K;
  constexpr bool later_singles = !MP, outer_pairs = !MP;
  const long long rstep = MP ? ((long long)R << s0) : (long long)R;  // element distance of consecutive cube rows
  const long long ngroups = d.dim >> K;
  // real s+ s- coefficients and warp-uniform row bits (a warp serves one cube)
  const bool real_fast = a.real_pm && (Rg % 32 == 0);

  // ---- per-system tables ----
  for (int q = threadIdx.x; q < n * n; q += bd) {
    const int i = q / n, j = q % n;
    if (i >= j) continue;
    const int ij = i * n + j, p = tri(i, j);
    const real pmr = t[L.off_pm + 2 * ij], pmi = t[L.off_pm + 2 * ij + 1];
    const real ppr = t[L.off_pp + 2 * ij], ppi = t[L.off_pp + 2 * ij + 1];
    real* c = S.cp + p * 8;
    c[0] = ppr; c[1] = -ppi;   // (0,0): mu = s-_i s-_j nu
    c[2] = pmr; c[3] = -pmi;   // (0,1): mu = s-_i s+_j nu
    c[4] = pmr; c[5] = pmi;    // (1,0): mu = s+_i s-_j nu
    c[6] = ppr; c[7] = ppi;    // (1,1): mu = s+_i s+_j nu
  }
  for (int q = threadIdx.x; q < n * NR; q += bd) {  // fcube[j][r] = sum_c rho_{j, s0+c} m_c(r)
    const int j = q / NR, r = q % NR;
    real fr = 0, fi = 0;
    for (int c = 0; c < K; ++c) {
      const real mc = ((r >> c) & 1) ? (real)0.5 : (real)-0.5;
      fr += t[L.off_rho + 2 * (j * n + s0 + c)] * mc;
      fi += t[L.off_rho + 2 * (j * n + s0 + c) + 1] * mc;
    }
    S.fcube[2 * q] = fr;
    S.fcube[2 * q + 1] = fi;
  }
  if (first) {  // the diagonal is done by the first pass, whose cube is bits [0, K)
    for (int r = threadIdx.x; r < NR; r += bd) {
      real e = 0;
      for (int c = 0; c < K; ++c) {
        const int bc = (r >> c) & 1;
        const real mc = bc ? (real)0.5 : (real)-0.5;
        e += t[L.off_hz + c] * mc + t[L.off_iondiag + c * L.qmax + bc];
        for (int c2 = c + 1; c2 < K; ++c2) e += t[L.off_zz + c * n + c2] * mc * (((r >> c2) & 1) ? (real)0.5 : (real)-0.5);
      }
      S.ecube[r] = e;
    }
  }

  double acc_d[4] = {0.0, 0.0, 0.0, 0.0};
  if (kPartials) {
    double* out = a.partials + (size_t)blockIdx.x * R * kNumPartials;
    for (int k = threadIdx.x; k < R * kNumPartials; k += bd) out[k] = 0.0;
  }
  int cur_vg = -1;
  real sig = 0, bsp = 0;
  const unsigned long long lowmask = (1ull << s0) - 1ull;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int vg = tile / a.tiles_per_vg;
    const long long g0 = (long long)(tile - vg * a.tiles_per_vg) * Gt;  // first cube of the tile
    const int k = vg * Rg + kl;
    const bool kvalid = k < R;
    if (vg != cur_vg) {
      if (kPartials && cur_vg >= 0) {  // flush the partials of the previous vector group
        __syncthreads();
        for (int c = 0; c < 4; ++c) S.red[threadIdx.x * 4 + c] = acc_d[c];
        __syncthreads();
        const int kk = cur_vg * Rg + threadIdx.x;
        if ((int)threadIdx.x < Rg && kk < R) {
          double sum[3] = {0, 0, 0};
          for (int sl = 0; sl < slots; ++sl)
            for (int c = 0; c < NPS; ++c) sum[c] += S.red[(threadIdx.x + sl * Rg) * 4 + c];
          double* out = a.partials + ((size_t)blockIdx.x * R + kk) * kNumPartials;
          for (int c = 0; c < NPS; ++c) out[c] = sum[c];
        }
        for (int c = 0; c < 4; ++c) acc_d[c] = 0.0;
      }
      if (MODE == kModeLanczos && kvalid) {
        sig = (real)d.sc.sigma[(size_t)a.step * d.sc.ss + k];
        bsp = a.first ? (real)0 : (real)(d.sc.beta[(size_t)(a.step - 1) * d.sc.ss + k] * d.sc.sigma[(size_t)(a.step - 1) * d.sc.ss + k]);
      }
      cur_vg = vg;
    }
    __syncthreads();  // the previous tile's cubes are done with fhi / ehi / gz
    // ---- per-tile outer parts ----
    const int fsites_lo = MP ? a.new_lo : 0, fsites_hi = MP ? s0 + K : n;  // sites whose single flips this pass does
    for (int q = threadIdx.x + fsites_lo * Gt; q < fsites_hi * Gt; q += bd) {
      const int j = q / Gt, g = q % Gt;
      const unsigned long long gi = (unsigned long long)(g0 + g);
      const unsigned long long mu0 = ((gi >> s0) << (s0 + K)) | (gi & lowmask);
      real fr = t[L.off_hp + 2 * j], fi = t[L.off_hp + 2 * j + 1];
      for (int i = 0; i < n; ++i) {
        if (i >= s0 && i < s0 + K) continue;
        const real mi = ((mu0 >> i) & 1ull) ? (real)0.5 : (real)-0.5;
        fr += t[L.off_rho + 2 * (j * n + i)] * mi;
        fi += t[L.off_rho + 2 * (j * n + i) + 1] * mi;
      }
      S.fhi[2 * q] = fr;
      S.fhi[2 * q + 1] = fi;
    }
    if (first) {
      for (int g = threadIdx.x; g < Gt; g += bd) {
        const unsigned long long mu0 = (unsigned long long)(g0 + g) << K;
        real e = 0;
        for (int i = K; i < n; ++i) {
          const int bi = (mu0 >> i) & 1ull;
          const real mi = bi ? (real)0.5 : (real)-0.5;
          real zs = t[L.off_hz + i];
          for (int j = i + 1; j < n; ++j) zs += t[L.off_zz + i * n + j] * (((mu0 >> j) & 1ull) ? (real)0.5 : (real)-0.5);
          e += mi * zs + t[L.off_iondiag + i * L.qmax + bi];
        }
        S.ehi[g] = e;
      }
      for (int q = threadIdx.x; q < K * Gt; q += bd) {
        const int c = q / Gt, g = q % Gt;
        const unsigned long long mu0 = (unsigned long long)(g0 + g) << K;
        real zs = 0;
        for (int i = K; i < n; ++i) zs += t[L.off_zz + c * n + i] * (((mu0 >> i) & 1ull) ? (real)0.5 : (real)-0.5);
        S.gz[q] = zs;
      }
    }
    __syncthreads();
    if (!kvalid) continue;
    real pacc[3] = {0, 0, 0};
    for (int g = slot; g < Gt; g += slots) {
      const long long gi = g0 + g;
      if (gi >= ngroups) break;  // ragged last tile
      const long long mu0 = (long long)((((unsigned long long)gi >> s0) << (s0 + K)) | ((unsigned long long)gi & lowmask));
      const void* x = d.x;
      const long long base = mu0 * R + k;
      v2 xo[NR];
      Cx<real> acc[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) xo[r] = ldx<real>(x, base + r * rstep);
      if (first) {  // diagonal
        const real eh = S.ehi[g];
        real gzc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) gzc[c] = S.gz[c * Gt + g];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          real e = eh + S.ecube[r];
#pragma unroll
          for (int c = 0; c < K; ++c) e += ((r >> c) & 1) ? (real)0.5 * gzc[c] : (real)-0.5 * gzc[c];
          acc[r].set(e, xo[r]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r].set((real)0, xo[r]);
      }
      // the pass's own cube bits: single flips and pairs, all in registers
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (c < cnew) continue;
        const int sc = s0 + c;
        const real fhr = S.fhi[2 * (sc * Gt + g)], fhim = S.fhi[2 * (sc * Gt + g) + 1];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const real fr = fhr + S.fcube[2 * (sc * NR + r)];
          const real fim = fhim + S.fcube[2 * (sc * NR + r) + 1];
          acc[r].mac(fr, ((r >> c) & 1) ? fim : -fim, xo[r ^ (1 << c)]);
        }
#pragma unroll
        for (int c1 = 0; c1 < c; ++c1) {
          if (c1 < cnew) continue;
          const real* cp = S.cp + tri(s0 + c1, sc) * 8;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const int idx = 2 * ((r >> c1) & 1) + ((r >> c) & 1);
            acc[r].mac(cp[2 * idx], cp[2 * idx + 1], xo[r ^ (1 << c) ^ (1 << c1)]);
          }
        }
      }
      // later bit j: the neighbouring cube serves the mixed pairs (c, j) (and, in the
      // single-pass form, the single flip of j)
      for (int j = later_lo; j < n; ++j) {
        const int bj = (int)((mu0 >> j) & 1);
        const long long nbase = (mu0 ^ (1ll << j)) * R + k;
        v2 y[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r] = ldx<real>(x, nbase + r * rstep);
        if (later_singles) {
          const real fhr = S.fhi[2 * (j * Gt + g)], fhim = S.fhi[2 * (j * Gt + g) + 1];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const real fr = fhr + S.fcube[2 * (j * NR + r)];
            const real fim = fhim + S.fcube[2 * (j * NR + r) + 1];
            acc[r].mac(fr, bj ? fim : -fim, y[r]);
          }
        }
#pragma unroll
        for (int c = 0; c < K; ++c) {
          if (c < cnew) continue;
          const real* cp = S.cp + tri(s0 + c, j) * 8;
          const real c0r = cp[2 * bj], c0i = cp[2 * bj + 1];            // bit c of the row = 0
          const real c1r = cp[2 * (2 + bj)], c1i = cp[2 * (2 + bj) + 1];  // bit c of the row = 1
          if (real_fast) {  // one of the two is an s+ s- coefficient: real
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              const int bc = (r >> c) & 1;
              if (bc != bj) acc[r].mac_re(bc ? c1r : c0r, y[r ^ (1 << c)]);
              else acc[r].mac(bc ? c1r : c0r, bc ? c1i : c0i, y[r ^ (1 << c)]);
            }
          } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              if ((r >> c) & 1) acc[r].mac(c1r, c1i, y[r ^ (1 << c)]);
              else acc[r].mac(c0r, c0i, y[r ^ (1 << c)]);
            }
          }
        }
      }
      // pairs among the later bits (single-pass form): one coefficient for the whole cube
      if (outer_pairs) {
        for (int j = later_lo + 1; j < n; ++j) {
          const int bj = (int)((mu0 >> j) & 1);
          const real* cpj = S.cp + tri(later_lo, j) * 8 + 2 * bj;
#pragma unroll 2
          for (int i = later_lo; i < j; ++i) {
            const int bi = (int)((mu0 >> i) & 1);
            const real* cp = cpj + (i - later_lo) * 8 + 4 * bi;
            const real cr = cp[0], ci = cp[1];
            const long long nbase = (mu0 ^ (1ll << j) ^ (1ll << i)) * R + k;
            v2 y[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) y[r] = ldx<real>(x, nbase + r * rstep);
            if (real_fast && bi != bj) {
#pragma unroll
              for (int r = 0; r < NR; ++r) acc[r].mac_re(cr, y[r]);
            } else {
#pragma unroll
              for (int r = 0; r < NR; ++r) acc[r].mac(cr, ci, y[r]);
            }
          }
        }
      }
      // epilogue
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const long long idx = base + r * rstep;
        v2 hv = acc[r].value();
        v2* yp = reinterpret_cast<v2*>(d.y) + idx;
        if (MODE == kModeApply) {
          if (!first) {
            const v2 prev = __ldcs(yp);
            hv.x += prev.x;
            hv.y += prev.y;
          }
          __stcs(yp, hv);
          if (kPartials) {  // Re <x|Hx>; the own rows are re-read (L1) rather than kept in registers
            const v2 xv = ldx<real>(x, idx);
            pacc[0] += xv.x * hv.x + xv.y * hv.y;
          }
        } else {
          v2 w;
          w.x = sig * hv.x;
          w.y = sig * hv.y;
          if (!a.first) {
            const v2 q = __ldcs(yp);
            w.x = fma(-bsp, q.x, w.x);
            w.y = fma(-bsp, q.y, w.y);
          }
          __stcs(yp, w);
          const v2 u = __ldcs(reinterpret_cast<const v2*>(d.u) + idx);
          const real vr = sig * xo[r].x, vi = sig * xo[r].y;
          pacc[0] += vr * w.x + vi * w.y;
          pacc[1] += vr * u.x + vi * u.y;
          pacc[2] += vr * u.y - vi * u.x;
        }
      }
    }
    if (kPartials)
      for (int c = 0; c < NPS; ++c) acc_d[c] += (double)pacc[c];
  }
  if (!kPartials) return;
  if (cur_vg >= 0) {
    __syncthreads();
    for (int c = 0; c < 4; ++c) S.red[threadIdx.x * 4 + c] = acc_d[c];
    __syncthreads();
    const int kk = cur_vg * Rg + threadIdx.x;
    if ((int)threadIdx.x < Rg && kk < R) {
      double sum[3] = {0, 0, 0};
      for (int sl = 0; sl < slots; ++sl)
        for (int c = 0; c < NPS; ++c) sum[c] += S.red[(threadIdx.x + sl * Rg) * 4 + c];
      double* out = a.partials + ((size_t)blockIdx.x * R + kk) * kNumPartials;
      for (int c = 0; c < NPS; ++c) out[c] = sum[c];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize(a, a.inline_one ? &a.one : a.inst);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---------------------------------------------------------------------------
template <typename real, int K, int RS, int MINB>
static int launch_krs(const LaunchArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  if (a.mode != kModeApply) return (int)cudaErrorInvalidValue;  // the Lanczos step runs the gather alone
  half_kernel<real, K, kModeApply, RS, false, MINB><<<grid, threads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename real, int K>
static int launch_k(const LaunchArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  if (a.mode != kModeApply) return (int)cudaErrorInvalidValue;
  if (!a.single_pass) {  // one pass of the multi-pass form
    half_kernel<real, K, kModeApply, 0, true, 1><<<grid, threads, smem, st>>>(a);
    return (int)cudaGetLastError();
  }
  if (a.min_blocks > 2) {
    if (a.R == 64) return launch_krs<real, K, 64, 3>(a, grid, threads, smem, st);
    return launch_krs<real, K, 0, 3>(a, grid, threads, smem, st);
  }
  if (a.R == 64) return launch_krs<real, K, 64, 2>(a, grid, threads, smem, st);
  return launch_krs<real, K, 0, 2>(a, grid, threads, smem, st);
}

int launch_half(const LaunchArgs& a, int K, int c64, int grid, int threads, size_t smem, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (c64) {
    switch (K) {
      case 2: return launch_k<float, 2>(a, grid, threads, smem, st);
      case 3: return launch_k<float, 3>(a, grid, threads, smem, st);
      case 4: return launch_k<float, 4>(a, grid, threads, smem, st);
    }
  } else {
    switch (K) {
      case 2: return launch_k<double, 2>(a, grid, threads, smem, st);
      case 3: return launch_k<double, 3>(a, grid, threads, smem, st);
      case 4: return launch_k<double, 4>(a, grid, threads, smem, st);
    }
  }
  return (int)cudaErrorInvalidValue;
}

template <typename real, int K>
static int allow_half(int bytes) {
  const void* ks[] = {(const void*)half_kernel<real, K, kModeApply, 0, false, 2>,
                      (const void*)half_kernel<real, K, kModeApply, 64, false, 2>,
                      (const void*)half_kernel<real, K, kModeApply, 0, false, 3>,
                      (const void*)half_kernel<real, K, kModeApply, 64, false, 3>,
                      (const void*)half_kernel<real, K, kModeApply, 0, true, 1>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

int prepare_half_kernels(size_t smem) {
  int e = allow_half<float, 2>((int)smem);
  if (!e) e = allow_half<float, 3>((int)smem);
  if (!e) e = allow_half<float, 4>((int)smem);
  if (!e) e = allow_half<double, 2>((int)smem);
  if (!e) e = allow_half<double, 3>((int)smem);
  if (!e) e = allow_half<double, 4>((int)smem);
  return e;
}

// Occupancy of the instantiation launch_k would pick for these arguments.
template <typename real, int K>
static int occ(int threads, size_t smem, int min_blocks, bool mp, int R) {
  int nb = 0;
  cudaError_t e;
  if (mp) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, half_kernel<real, K, kModeApply, 0, true, 1>, threads, smem);
  else if (min_blocks > 2 && R == 64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, half_kernel<real, K, kModeApply, 64, false, 3>, threads, smem);
  else if (min_blocks > 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, half_kernel<real, K, kModeApply, 0, false, 3>, threads, smem);
  else if (R == 64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, half_kernel<real, K, kModeApply, 64, false, 2>, threads, smem);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, half_kernel<real, K, kModeApply, 0, false, 2>, threads, smem);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int half_max_ctas_per_sm(int K, int c64, int threads, size_t smem, int min_blocks, bool multipass, int R) {
  if (c64) {
    if (K == 2) return occ<float, 2>(threads, smem, min_blocks, multipass, R);
    if (K == 3) return occ<float, 3>(threads, smem, min_blocks, multipass, R);
    return occ<float, 4>(threads, smem, min_blocks, multipass, R);
  }
  if (K == 2) return occ<double, 2>(threads, smem, min_blocks, multipass, R);
  if (K == 3) return occ<double, 3>(threads, smem, min_blocks, multipass, R);
  return occ<double, 4>(threads, smem, min_blocks, multipass, R);
}

}  // namespace ftlm
