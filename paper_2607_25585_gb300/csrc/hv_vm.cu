// Vector-major spin-1/2 H.v (Eq. 3 of arxiv 2607.25585 with every s_i = 1/2)
// for the Lanczos runs.
//
// Layout.  Every vector of the run is a contiguous array of d complex values
// (each vector is its own instance of the launch), so a vector's whole
// gathered slice -- d * 8 bytes in complex64, 8 MB at d = 2^20 -- stays in L2
// while its neighbours are read, and a warp's loads are 32 consecutive rows.
//
// Thread mapping.  The 32 lanes of a warp hold 32 consecutive rows (bits
// 0..4 of the row index); each thread owns a register cube along bits
// [5, 5 + K) for its lane, i.e. 2^K rows of one vector; a warp processes one
// slab of 2^(5+K) consecutive rows at a time.  Flips of cube bits read
// registers; every other bit (the lane bits and the slab bits above the cube)
// is gathered as in the low-bit register-cube kernel: one neighbouring cube
// per bit j serves the single flip of j and the K mixed pairs (c, j), one per
// pair of outer bits.  Flips of the lane bits and of the low slab bits land in
// rows the same CTA has just read (L1).
//
// Coefficients.  The single-flip coefficient of site j and the diagonal are
// sums over bit groups: lane bits (per-system tables indexed by the lane),
// cube bits (tables indexed by the cube row) and slab bits (computed per slab
// by the warp's lanes in parallel).
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"

namespace ftlm {

namespace {

constexpr int kLaneBits = kVmLaneBits;

// x[base + r * 2^s0]: in the single-pass form (s0 = 5 at compile time) a
// 64-bit base with constant offsets; in the multi-pass form (s0 from the pass)
// 32-bit element indices (the vector-major kernels require d < 2^31)
template <typename real, bool MP>
__device__ __forceinline__ typename Cx<real>::v2 ldx_cube(const void* x, long long base, int r, int s0) {
  using v2 = typename Cx<real>::v2;
  if (MP) return __ldg(reinterpret_cast<const v2*>(x) + ((unsigned)base + ((unsigned)r << s0)));
  return __ldg(reinterpret_cast<const v2*>(x) + base + ((long long)r << s0));
}

template <typename real>
struct VmSmem {
  real* cp;   // [npairs][4][2] pair coefficients by (bit_i, bit_j) of the row
  real* cpl;  // the same with the pairs of the last pass's overlap bits zeroed (multi-pass)
  real* fl;   // [n][32][2]  sum_{i < 5} rho_ji m_i(lane)
  real* fc;   // [npass][n][NR][2]  sum_c rho_{j, s0(p)+c} m_c(r), cube of pass p
  real* el;   // [32]        diagonal from the lane bits alone
  real* gl;   // [K][32]     sum_{i < 5} zz_{i, 5+c} m_i(lane)
  real* ec;   // [NR]        diagonal from the cube bits alone (first pass)
  real* ws;   // per warp: fs [n][2], hs [5], gs [K], es [1]
};

template <typename real>
__device__ VmSmem<real> vm_carve(unsigned char* raw, int n, int K, int npass, int& warp_stride) {
  VmSmem<real> s;
  const int NR = 1 << K;
  const int npairs = n * (n - 1) / 2;
  real* p = reinterpret_cast<real*>(raw);
  s.cp = p;
  p += npairs * 8;
  s.cpl = s.cp;
  if (npass > 1) {  // the last pass's table with the overlap bits zeroed
    s.cpl = p;
    p += npairs * 8;
  }
  s.fl = p;
  p += n * 32 * 2;
  s.fc = p;
  p += npass * n * NR * 2;
  s.el = p;
  p += 32;
  s.gl = p;
  p += K * 32;
  s.ec = p;
  p += NR;
  s.ws = p;
  warp_stride = (2 * n + kLaneBits + K + 1 + 1) & ~1;  // even: each warp's fs starts at a pair boundary
  return s;
}

// a (re, im) pair of a shared-memory table as one 8- or 16-byte access (the
// tables keep every pair at an even offset from a 16-byte-aligned base)
template <typename real>
__device__ __forceinline__ typename Cx<real>::v2 ld2(const real* p) {
  return *reinterpret_cast<const typename Cx<real>::v2*>(p);
}

// zz coefficient of sites (i, j), stored for i < j
template <typename real>
__device__ __forceinline__ real zzc(const real* t, const TabLayout& L, int n, int i, int j) {
  return i < j ? t[L.off_zz + i * n + j] : t[L.off_zz + j * n + i];
}

__host__ __device__ constexpr int ctz_const(int x) {
  int c = 0;
  while (!(x & 1)) {
    x >>= 1;
    ++c;
  }
  return c;
}

// The cube-dependent part of site j's single-flip coefficient,
// fc(r) = sum_c rho_{j, cube bit c} m_c(r), for the 2^K cube rows r in
// Gray-code order (consecutive rows differ in one bit c, so fc changes by
// +-rho_c): f(r, fc(r)) for every r, from 1 + K shared-memory reads of the
// table fcp_j[r] (rows 0 and 2^c) instead of 2^K.
template <typename real, int K, typename F>
__device__ __forceinline__ void gray_fc(const real* fcp_j, F&& f) {
  using v2 = typename Cx<real>::v2;
  constexpr int NR = 1 << K;
  const v2 f0 = *reinterpret_cast<const v2*>(fcp_j);
  v2 rho[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const v2 fb = *reinterpret_cast<const v2*>(fcp_j + 2 * (1 << c));
    rho[c].x = fb.x - f0.x;
    rho[c].y = fb.y - f0.y;
  }
  v2 v = f0;
#pragma unroll
  for (int g = 0; g < NR; ++g) {
    f(g ^ (g >> 1), v);
    if (g + 1 < NR) {
      const int c = ctz_const(g + 1);
      if ((((g + 1) ^ ((g + 1) >> 1)) >> c) & 1) {
        v.x += rho[c].x;
        v.y += rho[c].y;
      } else {
        v.x -= rho[c].x;
        v.y -= rho[c].y;
      }
    }
  }
}

}  // namespace

// Dynamic shared memory of vm_kernel (tables of `real`: 4 bytes for
// complex64, 8 for complex128).  Kept small: the rest of the SM's 256 KB of
// L1/shared memory is L1 cache, which serves most gathered loads.
size_t vm_smem_bytes(int n, int K, int threads, int npass, int c64) {
  const int NR = 1 << K, nwarps = threads / 32;
  const size_t reals = (size_t)(n * (n - 1) / 2) * 8 * (npass > 1 ? 2 : 1) + (size_t)n * 32 * 2 +
                       (size_t)npass * n * NR * 2 + 32 + (size_t)K * 32 + NR +
                       (size_t)nwarps * ((2 * n + kLaneBits + K + 2) & ~1);
  return reals * (c64 ? 4 : 8);
}

// Cube of pass p of the multi-pass form: bits [s0, s0 + K) with s0 = min(5 + pK, n - K);
// its own bits start at 5 + pK (the last cube may overlap the one before).
__device__ __forceinline__ int vm_pass_lo(int p, int K, int n) { return min(kLaneBits + p * K, n - K); }

// The two-pass form, two launches (a.hybrid): launch 1 is the one-pass kernel
// (cube on bits [5, 5 + K)) doing everything except the terms of the top K
// bits (a.hybrid = 1); launch 2 (a.hybrid = 2, multi-pass template) has its
// cube on the top bits [n - K, n) and does their single flips, their pairs
// with each other and their mixed pairs with the lane bits and the middle bits
// [5 + K, n - K), adds the first launch's sums and writes the complete H x.
// Pairs of a bottom-cube bit with a top bit are mixed pairs of launch 1.

// MP: the multi-pass form, all a.npass passes in this launch.  Pass p's cube
// spans bits [s0, s0 + K), s0 = min(5 + pK, n - K); its cube bits >= 5 + pK
// are its own: their single flips, their pairs with each other and their
// mixed pairs with the lane bits and with the bits above the cube.  Pass 0
// (cube on bits [5, 5 + K)) also does the diagonal, the lane bits' single
// flips and the lane-lane pairs.  Every pair is then a cube pair, a mixed
// pair or a lane-lane pair of exactly one pass, so each gathered load serves
// K (or K + 1) multiply-adds per row instead of one.  Pass p writes its
// partial H x to y + p * a.pass_stride; the consumer adds the a.npass blocks in
// pass order.  Tiles run vector by vector, the passes of a vector side by side,
// so a vector's x is read from HBM once and then served from L2.
// Without MP: one pass, cube on bits [5, 5 + K), every term; pairs of two bits
// outside the cube cost one gathered load per multiply-add.
// MINB: resident CTAs per SM the register allocator must allow: 2 or 3 CTAs
// of 256 threads, or 1 = one CTA of 512 threads (the same registers per
// thread as 2; one copy of the tables per SM leaves more of it to L1).
template <typename real, int K, bool MP, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? 512 : 256, MINB) vm_kernel(const __grid_constant__ LaunchArgs a) {
  using v2 = typename Cx<real>::v2;
  constexpr int NR = 1 << K;
  constexpr int CB = kLaneBits;  // lane bits [0, CB)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDesc d;
  __shared__ double wacc[16][3];  // per warp: its units' partial sums for the current vector (FP64)
  __shared__ double s_sg, s_bsp;  // fused step: sigma_j and beta_j sigma_{j-1} of the current vector
  __shared__ const void* s_u;     // fused step: the current vector's observable block
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool kPartials = a.gather_alpha != 0 || a.fused_step != 0;  // Re<x|Hx> (or <x|w'>, <x|u>) per vector
  const bool fused = !MP && a.fused_step != 0;  // the step's w' in the epilogue (one-pass form only)
  const InstDesc* insts = a.inline_one ? &a.one : a.inst;
  if (threadIdx.x == 0) d = insts[0];
  for (int k = threadIdx.x; k < 16 * 3; k += blockDim.x) wacc[k / 3][k % 3] = 0.0;
  __syncthreads();
  const int n = d.n;
  const int P = MP ? a.npass : 1;
  int wstride = 0;
  const VmSmem<real> S = vm_carve<real>(smem_raw, n, K, P, wstride);
  const real* t = reinterpret_cast<const real*>(d.tab);  // every instance of the launch shares the system
  const TabLayout& L = d.lay;
  const int bd = blockDim.x;
  const bool top = MP && a.hybrid == 2;       // the top-cube launch of the two-pass form
  const bool bottom = !MP && a.hybrid == 1;   // the bottom-cube launch of the two-pass form
  // cube of pass p: bits [cube_lo(p), cube_lo(p) + K)
  auto cube_lo = [&](int p) { return top ? n - K : vm_pass_lo(p, K, n); };
  // the last pass's cube bits below its own bits (overlap with the pass before)
  const int ov_lo = vm_pass_lo(P - 1, K, n), ov_hi = (MP && !top) ? CB + (P - 1) * K : ov_lo;
  auto overlap = [&](int i) { return i >= ov_lo && i < ov_hi; };

  // ---- per-system tables ----
  for (int q = threadIdx.x; q < n * n; q += bd) {
    const int i = q / n, j = q % n;
    if (i >= j) continue;
    const int ij = i * n + j;
    const real pmr = t[L.off_pm + 2 * ij], pmi = t[L.off_pm + 2 * ij + 1];
    const real ppr = t[L.off_pp + 2 * ij], ppi = t[L.off_pp + 2 * ij + 1];
    real* c = S.cp + tri(i, j) * 8;
    c[0] = ppr; c[1] = -ppi;   // (0,0): mu = s-_i s-_j nu
    c[2] = pmr; c[3] = -pmi;   // (0,1): mu = s-_i s+_j nu
    c[4] = pmr; c[5] = pmi;    // (1,0): mu = s+_i s-_j nu
    c[6] = ppr; c[7] = ppi;    // (1,1): mu = s+_i s+_j nu
    real* cl = S.cpl + tri(i, j) * 8;
    const real z = (overlap(i) || overlap(j)) ? (real)0 : (real)1;
    for (int k = 0; k < 8; ++k) cl[k] = z * c[k];
  }
  for (int q = threadIdx.x; q < n * 32; q += bd) {  // lane part of F_j
    const int j = q / 32, l = q % 32;
    real fr = 0, fi = 0;
    for (int i = 0; i < CB; ++i) {
      const real mi = ((l >> i) & 1) ? (real)0.5 : (real)-0.5;
      fr += t[L.off_rho + 2 * (j * n + i)] * mi;
      fi += t[L.off_rho + 2 * (j * n + i) + 1] * mi;
    }
    S.fl[2 * q] = fr;
    S.fl[2 * q + 1] = fi;
  }
  for (int q = threadIdx.x; q < P * n * NR; q += bd) {  // cube part of F_j, per pass
    const int pp = q / (n * NR), j = (q / NR) % n, r = q % NR;
    const int c0 = MP ? cube_lo(pp) : CB;
    real fr = 0, fi = 0;
    if (!(pp == P - 1 && overlap(j))) {
      for (int c = 0; c < K; ++c) {
        const real mc = ((r >> c) & 1) ? (real)0.5 : (real)-0.5;
        fr += t[L.off_rho + 2 * (j * n + c0 + c)] * mc;
        fi += t[L.off_rho + 2 * (j * n + c0 + c) + 1] * mc;
      }
    }
    S.fc[2 * q] = fr;
    S.fc[2 * q + 1] = fi;
  }
  for (int l = threadIdx.x; l < 32; l += bd) {  // lane bits: diagonal and cross terms with the first cube
    real e = 0;
    for (int i = 0; i < CB; ++i) {
      const int bi = (l >> i) & 1;
      const real mi = bi ? (real)0.5 : (real)-0.5;
      e += t[L.off_hz + i] * mi + t[L.off_iondiag + i * L.qmax + bi];
      for (int i2 = i + 1; i2 < CB; ++i2) e += zzc(t, L, n, i, i2) * mi * (((l >> i2) & 1) ? (real)0.5 : (real)-0.5);
    }
    S.el[l] = e;
    for (int c = 0; c < K; ++c) {
      real g = 0;
      for (int i = 0; i < CB; ++i) g += zzc(t, L, n, i, CB + c) * (((l >> i) & 1) ? (real)0.5 : (real)-0.5);
      S.gl[c * 32 + l] = g;
    }
  }
  for (int r = threadIdx.x; r < NR; r += bd) {  // first cube's bits alone
    real e = 0;
    for (int c = 0; c < K; ++c) {
      const int bc = (r >> c) & 1;
      const real mc = bc ? (real)0.5 : (real)-0.5;
      e += t[L.off_hz + CB + c] * mc + t[L.off_iondiag + (CB + c) * L.qmax + bc];
      for (int c2 = c + 1; c2 < K; ++c2)
        e += zzc(t, L, n, CB + c, CB + c2) * mc * (((r >> c2) & 1) ? (real)0.5 : (real)-0.5);
    }
    S.ec[r] = e;
  }
  __syncthreads();

  real* W = S.ws + warp * wstride;  // this warp's unit tables
  real* fs = W;                     // [n][2]
  real* hs = W + 2 * n;             // [5]
  real* gs = hs + CB;               // [K]
  real* es = gs + K;                // [1]
  // a unit: 32 lanes x the cube = 2^(5+K) rows whose other ("outer") bits are fixed
  const long long nunits = d.dim >> (CB + K);
  const int units_per_tile = a.rows_per_tile >> (CB + K);
  const bool real_fast_pm = a.real_pm != 0;
  if (kPartials)  // this CTA's slot of every vector: [vector][CTA][kNumPartials]
    for (int k = threadIdx.x; k < a.n_inst * kNumPartials; k += bd)
      a.partials[((size_t)(k / kNumPartials) * gridDim.x + blockIdx.x) * kNumPartials + k % kNumPartials] = 0.0;
  // Partial sums, in a fixed order: each thread's sums over its rows of a unit
  // are added across the warp in FP64 (the Lanczos scalars need FP64 sums:
  // alpha_j and p_j feed the Ritz values and weights) and into the warp's FP64
  // slot; flush adds the slots of the CTA's warps for vector `inst`.
  // Re<x|Hx> (gather_alpha), or Re<x|w'>, Re<x|u>, Im<x|u> (fused step).
  const int np = fused ? 3 : 1;
  auto add_unit = [&](real p0f, real p1f, real p2f) {
    double p0 = (double)p0f, p1 = (double)p1f, p2 = (double)p2f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, o);
      if (fused) {
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
      }
    }
    if (lane == 0) {
      wacc[warp][0] += p0;
      if (fused) {
        wacc[warp][1] += p1;
        wacc[warp][2] += p2;
      }
    }
  };
  auto flush = [&](int inst) {
    __syncthreads();
    if (threadIdx.x < np) {  // the sum over the warps, then the slots start again from zero
      double tot = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        tot += wacc[w][threadIdx.x];
        wacc[w][threadIdx.x] = 0.0;
      }
      a.partials[((size_t)inst * gridDim.x + blockIdx.x) * kNumPartials + threadIdx.x] = tot;
    }
    __syncthreads();
  };
  int cur = -1;
  const void* x = nullptr;
  void* y0 = nullptr;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    // tiles: [vector][pass][tile of the pass]
    const int inst = tile / (P * a.tiles_per_vg);
    const int pass = MP ? (tile / a.tiles_per_vg) % P : 0;
    const int ptile = tile % a.tiles_per_vg;
    if (inst != cur) {  // per-vector pointers (the tables are shared)
      if (kPartials && cur >= 0) flush(cur);
      if (fused) {
        __syncthreads();  // every warp is done with the previous vector's scalars
        if (threadIdx.x == 0) {
          const DevScalars& sc = insts[inst].sc;
          const int j = a.step;
          s_sg = sc.sigma[(size_t)j * sc.ss];
          s_bsp = a.first ? 0.0 : sc.beta[(size_t)(j - 1) * sc.ss] * sc.sigma[(size_t)(j - 1) * sc.ss];
          s_u = insts[inst].u;
        }
        __syncthreads();
      }
      if (a.vm_stride) {  // a regular vector-major block: vector inst at a fixed stride
        x = static_cast<const char*>(a.one.x) + (long long)inst * a.vm_stride;
        y0 = static_cast<char*>(a.one.y) + (long long)inst * a.vm_stride;
      } else {
        x = insts[inst].x;
        y0 = insts[inst].y;
      }
      cur = inst;
    }
    const int s0 = MP ? cube_lo(pass) : CB;                 // cube bits [s0, s0 + K)
    const int cnew = (MP && !top) ? CB + pass * K - s0 : 0;  // first own cube bit (cube-relative)
    const bool first = !MP || (pass == 0 && !top);
    // neighbour bits: the lane bits and [nb_lo, nb_hi) (the bits above the cube,
    // or for the top cube of the two-pass form the middle bits below it)
    const int nb_lo = top ? CB + K : s0 + K;
    const int nb_hi = top ? s0 : n;
    // single flips of neighbour bits below single_hi and pairs of two neighbour
    // bits below pair_hi belong to this pass (only in the first pass)
    const int single_hi = !MP ? (bottom ? n - K : n) : CB;
    const int pair_hi = single_hi;
    const real* cpb = (MP && pass == P - 1) ? S.cpl : S.cp;  // overlap pairs zeroed in the last pass
    const real* fcp = S.fc + (size_t)pass * n * NR * 2;
    v2* const y = reinterpret_cast<v2*>(y0) + (MP ? pass * a.pass_stride : 0);
    const unsigned long long lowmask = (1ull << (s0 - CB)) - 1ull;  // outer bits between the lanes and the cube
    const int nnb = CB + nb_hi - nb_lo;
    auto in_cube = [&](int i) { return i >= s0 && i < s0 + K; };
    const long long unit0 = (long long)ptile * units_per_tile;
    for (int ui = warp; ui < units_per_tile; ui += nwarps) {
      const unsigned long long u = (unsigned long long)(unit0 + ui);
      if ((long long)u >= nunits) break;
      const unsigned long long base = ((u >> (s0 - CB)) << (s0 + K)) | ((u & lowmask) << CB);
      // unit tables (the outer bits' share of the coefficients): copied from the
      // system's precomputed per-unit tables (one-pass form), or built by the
      // warp's lanes in parallel
      __syncwarp();
      const bool from_table = !MP && a.hybrid == 0 && a.unit_tab != nullptr;
      if (from_table) {
        const real* src = reinterpret_cast<const real*>(a.unit_tab) + (size_t)u * wstride;
        for (int k = lane; k < wstride; k += 32) W[k] = src[k];
      }
      for (int j = lane; j < n && !from_table; j += 32) {
        real fr = t[L.off_hp + 2 * j], fi = t[L.off_hp + 2 * j + 1];
        for (int i = CB; i < n; ++i) {
          if (in_cube(i)) continue;
          const real mi = ((base >> i) & 1ull) ? (real)0.5 : (real)-0.5;
          fr += t[L.off_rho + 2 * (j * n + i)] * mi;
          fi += t[L.off_rho + 2 * (j * n + i) + 1] * mi;
        }
        fs[2 * j] = fr;
        fs[2 * j + 1] = fi;
      }
      if (first && !from_table) {
        if (lane < CB) {  // lane bit `lane` x outer bits
          real h = 0;
          for (int j = CB; j < n; ++j)
            if (!in_cube(j)) h += zzc(t, L, n, lane, j) * (((base >> j) & 1ull) ? (real)0.5 : (real)-0.5);
          hs[lane] = h;
        } else if (lane < CB + K) {  // cube bit x outer bits
          const int c = lane - CB;
          real g = 0;
          for (int i = CB; i < n; ++i)
            if (!in_cube(i)) g += zzc(t, L, n, s0 + c, i) * (((base >> i) & 1ull) ? (real)0.5 : (real)-0.5);
          gs[c] = g;
        }
        // diagonal of the outer bits alone: lane i adds the terms of outer bit i
        // (Zeeman, single-ion, zz with the outer bits above i), then a warp sum
        real e = 0;
        for (int i = lane; i < n; i += 32) {
          if (i < CB || in_cube(i)) continue;
          const int bi = (base >> i) & 1ull;
          real zs = t[L.off_hz + i];
          for (int j = i + 1; j < n; ++j)
            if (!in_cube(j)) zs += zzc(t, L, n, i, j) * (((base >> j) & 1ull) ? (real)0.5 : (real)-0.5);
          e += (bi ? (real)0.5 : (real)-0.5) * zs + t[L.off_iondiag + i * L.qmax + bi];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) es[0] = e;
      }
      __syncwarp();
      const long long row0 = (long long)(base | (unsigned long long)lane);
      if (fused) {  // the epilogue's own rows of q_{j-1} and u to L2 while the unit is gathered
        const v2* uu = reinterpret_cast<const v2*>(s_u);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const long long e = row0 + ((long long)r << s0);
          if (!a.first) asm volatile("prefetch.global.L2 [%0];" ::"l"(y + e));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(uu + e));
        }
      }
      if (MP && ui + nwarps < units_per_tile && (long long)u + nwarps < nunits) {
        // the warp's next unit: its rows of x (and of y for the top launch) to L2 now,
        // so that the unit's first loads do not wait on HBM
        const unsigned long long un = u + (unsigned long long)nwarps;
        const unsigned long long bn = ((un >> (s0 - CB)) << (s0 + K)) | ((un & lowmask) << CB) | (unsigned long long)lane;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const v2*>(x) + ((unsigned)bn + ((unsigned)r << s0))));
          if (top) asm volatile("prefetch.global.L2 [%0];" ::"l"(y + ((unsigned)bn + ((unsigned)r << s0))));
        }
      }
      v2 xo[NR];
      Cx<real> acc[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) xo[r] = ldx_cube<real, MP>(x, row0, r, s0);
      if (first) {  // diagonal
        real eo = S.el[lane] + es[0];
#pragma unroll
        for (int i = 0; i < CB; ++i) eo += (((lane >> i) & 1) ? (real)0.5 : (real)-0.5) * hs[i];
        real g[K];
#pragma unroll
        for (int c = 0; c < K; ++c) g[c] = S.gl[c * 32 + lane] + gs[c];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          real e = eo + S.ec[r];
#pragma unroll
          for (int c = 0; c < K; ++c) e += ((r >> c) & 1) ? (real)0.5 * g[c] : (real)-0.5 * g[c];
          acc[r].set(e, xo[r]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r].set((real)0, xo[r]);
      }
      // own cube bits: single flips and pairs in registers (an overlap bit of the
      // last pass has zero coefficients)
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const int sc = s0 + c;
        const real om = (MP && c < cnew) ? (real)0 : (real)1;
        const v2 f0 = ld2(fs + 2 * sc), f1 = ld2(S.fl + 2 * (sc * 32 + lane));
        const real br = om * (f0.x + f1.x);
        const real bi = om * (f0.y + f1.y);
        if (!MP) {
          gray_fc<real, K>(fcp + 2 * (sc * NR), [&](int r, const v2 fc) {
            const real fim = bi + fc.y;
            acc[r].mac(br + fc.x, ((r >> c) & 1) ? fim : -fim, xo[r ^ (1 << c)]);
          });
        } else {
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const v2 fc = ld2(fcp + 2 * (sc * NR + r));
            const real fr = br + fc.x;
            const real fim = bi + fc.y;
            acc[r].mac(fr, ((r >> c) & 1) ? fim : -fim, xo[r ^ (1 << c)]);
          }
        }
#pragma unroll
        for (int c1 = 0; c1 < c; ++c1) {
          const real* cp = cpb + tri(s0 + c1, sc) * 8;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const int idx = 2 * ((r >> c1) & 1) + ((r >> c) & 1);
            const v2 cv = ld2(cp + 2 * idx);
            acc[r].mac(cv.x, cv.y, xo[r ^ (1 << c) ^ (1 << c1)]);
          }
        }
      }
      // neighbour bit j (a lane bit, or a bit above the cube): the neighbouring
      // cube serves the mixed pairs (c, j) and, where this pass owns it, the
      // single flip of j
      for (int jj = 0; jj < nnb; ++jj) {
        const int j = jj < CB ? jj : nb_lo + (jj - CB);
        const int bj = (int)((row0 >> j) & 1);
        const long long nb = row0 ^ (1ll << j);
        v2 yv[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) yv[r] = ldx_cube<real, MP>(x, nb, r, s0);
        if (first && j < single_hi) {
          const v2 f0 = ld2(fs + 2 * j), f1 = ld2(S.fl + 2 * (j * 32 + lane));
          const real br = f0.x + f1.x, bi = f0.y + f1.y;
          if (!MP) {
            gray_fc<real, K>(fcp + 2 * (j * NR), [&](int r, const v2 fc) {
              const real fim = bi + fc.y;
              acc[r].mac(br + fc.x, bj ? fim : -fim, yv[r]);
            });
          } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              const v2 fc = ld2(fcp + 2 * (j * NR + r));
              const real fim = bi + fc.y;
              acc[r].mac(br + fc.x, bj ? fim : -fim, yv[r]);
            }
          }
        }
        const bool uniform = j >= CB;  // bit j (not a lane bit) is the same for the whole warp
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const int sc = s0 + c;
          const bool lo = j < sc;
          // pair (min, max); its coefficients for the row's bit c = 0 and = 1 (bit j is bj)
          const real* cp = cpb + (lo ? tri(j, sc) : tri(sc, j)) * 8;
          const int i0 = lo ? 2 * bj : bj, i1 = lo ? 2 * bj + 1 : 2 + bj;
          const v2 cv0 = ld2(cp + 2 * i0), cv1 = ld2(cp + 2 * i1);
          const real c0r = cv0.x, c0i = cv0.y, c1r = cv1.x, c1i = cv1.y;
          if (uniform && real_fast_pm) {  // rows whose bit c differs from bj: the real s+ s- coefficient
            if (bj) {
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                if ((r >> c) & 1) acc[r].mac(c1r, c1i, yv[r ^ (1 << c)]);
                else acc[r].mac_re(c0r, yv[r ^ (1 << c)]);
              }
            } else {
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                if ((r >> c) & 1) acc[r].mac_re(c1r, yv[r ^ (1 << c)]);
                else acc[r].mac(c0r, c0i, yv[r ^ (1 << c)]);
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              if ((r >> c) & 1) acc[r].mac(c1r, c1i, yv[r ^ (1 << c)]);
              else acc[r].mac(c0r, c0i, yv[r ^ (1 << c)]);
            }
          }
        }
      }
      // pairs of two neighbour bits below pair_hi: one coefficient for the whole
      // cube (in one pass every such pair; in the multi-pass form only the
      // lane-lane pairs, in the two-pass form those of the lane and middle bits)
      if (first) {
        const int npb = CB + max(0, min(nb_hi, pair_hi) - nb_lo);
        for (int jj = 1; jj < npb; ++jj) {
          const int j = jj < CB ? jj : nb_lo + (jj - CB);
          const int bj = (int)((row0 >> j) & 1);
#pragma unroll 2
          for (int ii = 0; ii < jj; ++ii) {
            const int i = ii < CB ? ii : nb_lo + (ii - CB);
            const int bi = (int)((row0 >> i) & 1);
            const real* cp = cpb + tri(i, j) * 8 + 2 * (2 * bi + bj);
            const v2 cv = ld2(cp);
            const real cr = cv.x, ci = cv.y;
            const long long nb = row0 ^ (1ll << i) ^ (1ll << j);
            v2 yv[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) yv[r] = ldx_cube<real, MP>(x, nb, r, s0);
            if (i >= CB && real_fast_pm && bi != bj) {  // warp-uniform and real
#pragma unroll
              for (int r = 0; r < NR; ++r) acc[r].mac_re(cr, yv[r]);
            } else {
#pragma unroll
              for (int r = 0; r < NR; ++r) acc[r].mac(cr, ci, yv[r]);
            }
          }
        }
      }
      if (top) {  // add the bottom launch's sums: all loads first
        v2 prev[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) prev[r] = __ldcs(y + ((unsigned)row0 + ((unsigned)r << s0)));
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r].add(prev[r]);
      }
      if (fused) {  // w' = sigma_j H q_j - beta_j sigma_{j-1} q_{j-1} over q_{j-1}; <q_j|w'>, <q_j|u>
        const v2* uu = reinterpret_cast<const v2*>(s_u);
        const real sg = (real)s_sg, bsp = (real)s_bsp;
        real pw = 0, pur = 0, pui = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const long long e = row0 + ((long long)r << s0);
          const v2 hv = acc[r].value();
          v2 w;
          if (a.first) {
            w.x = sg * hv.x;
            w.y = sg * hv.y;
          } else {
            const v2 qp = __ldcs(y + e);
            w.x = sg * hv.x - bsp * qp.x;
            w.y = sg * hv.y - bsp * qp.y;
          }
          __stcs(y + e, w);
          const v2 xv = ldx_cube<real, MP>(x, row0, r, s0);  // own rows of q_j, re-read (L1)
          const v2 uv = __ldcs(uu + e);
          pw += xv.x * w.x + xv.y * w.y;
          pur += xv.x * uv.x + xv.y * uv.y;
          pui += xv.x * uv.y - xv.y * uv.x;
        }
        add_unit(pw, pur, pui);
      } else {
        real pd = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const v2 hv = acc[r].value();
          __stcs(MP ? y + ((unsigned)row0 + ((unsigned)r << s0)) : y + row0 + ((long long)r << s0), hv);
          if (kPartials) {  // the own rows are re-read (L1) rather than kept in registers
            const v2 xv = ldx_cube<real, MP>(x, row0, r, s0);
            pd += xv.x * hv.x + xv.y * hv.y;
          }
        }
        if (kPartials) add_unit(pd, (real)0, (real)0);
      }
    }
  }
  if (!kPartials) return;
  if (cur >= 0) flush(cur);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize(a, insts);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// Streaming modes (kModeStep, kModeStartNorm) on the vector-major block: R
// one-vector instances, tiles of a.rows_per_tile consecutive elements of one
// vector (a.tiles_per_vg per vector); a thread moves 16 bytes per array and
// item (two complex64 or one complex128 value).
template <typename real, int MODE>
__global__ void __launch_bounds__(256) vm_stream_kernel(const __grid_constant__ LaunchArgs a) {
  constexpr int V = sizeof(real) == 4 ? 2 : 1;
  __shared__ InstDesc d;
  __shared__ double red[32][kNumPartials];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int bd = blockDim.x;
  for (int k = threadIdx.x; k < a.n_inst * kNumPartials; k += bd)
    a.partials[((size_t)(k / kNumPartials) * gridDim.x + blockIdx.x) * kNumPartials + k % kNumPartials] = 0.0;
  double acc[3] = {0.0, 0.0, 0.0};
  auto flush = [&](int inst) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double v = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][c] = v;
      acc[c] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += red[w][threadIdx.x];
      a.partials[((size_t)inst * gridDim.x + blockIdx.x) * kNumPartials + threadIdx.x] = t;
    }
    __syncthreads();
  };
  int cur = -1;
  real sig[V], bsp[V], coef[V];
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int inst = tile / a.tiles_per_vg;
    if (inst != cur) {
      if (cur >= 0) flush(cur);
      {  // the instance's descriptor, copied by the whole CTA in 8-byte words
        static_assert(sizeof(InstDesc) % 8 == 0, "InstDesc is copied in 8-byte words");
        const long long* src = reinterpret_cast<const long long*>(a.inst + inst);
        long long* dst = reinterpret_cast<long long*>(&d);
        for (int w = threadIdx.x; w < (int)(sizeof(InstDesc) / 8); w += bd) dst[w] = __ldg(src + w);
      }
      __syncthreads();
      const int j = a.step;
      real sg = 0, bs = 0, cf = 0;
      if (MODE == kModeStep) {
        sg = (real)d.sc.sigma[(size_t)j * d.sc.ss];
        if (!a.first) bs = (real)(d.sc.beta[(size_t)(j - 1) * d.sc.ss] * d.sc.sigma[(size_t)(j - 1) * d.sc.ss]);
        cf = (real)(d.sc.alpha[(size_t)j * d.sc.ss] * d.sc.sigma[(size_t)j * d.sc.ss]);
      } else if (MODE == kModeUpdate) {  // the tail of the fused step: w = w' - alpha_j sigma_j q_j
        cf = (real)(d.sc.alpha[(size_t)j * d.sc.ss] * d.sc.sigma[(size_t)j * d.sc.ss]);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sig[v] = sg;
        bsp[v] = bs;
        coef[v] = cf;
      }
      cur = inst;
    }
    const long long e0 = (long long)(tile - inst * a.tiles_per_vg) * a.rows_per_tile;
    const long long e_end = min(e0 + (long long)a.rows_per_tile, d.dim);
    real pacc[V * kNumPartials];
#pragma unroll
    for (int k = 0; k < V * kNumPartials; ++k) pacc[k] = 0;
    const long long step = (long long)bd * V;
    long long e = e0 + (long long)threadIdx.x * V;
    if (MODE == kModeStep) {
      step_stream<real, V, 4>(d, a, e, e_end, step, sig, bsp, coef, pacc);
    } else if (MODE == kModeUpdate) {
      update_stream<real, V, 4>(d, e, e_end, step, coef, pacc);
    } else {
      for (; e + step < e_end; e += 2 * step) {
        elementwise_item<real, V, MODE>(d, a, e, sig, bsp, coef, pacc);
        elementwise_item<real, V, MODE>(d, a, e + step, sig, bsp, coef, pacc);
      }
      if (e < e_end) elementwise_item<real, V, MODE>(d, a, e, sig, bsp, coef, pacc);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      real t = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) t += pacc[v * kNumPartials + c];
      acc[c] += (double)t;
    }
  }
  if (cur >= 0) flush(cur);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize(a, a.inst);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// The per-unit tables of the one-pass vector-major gather (cube on bits
// [5, 5 + K), outer bits [5 + K, n)): for unit u (outer bits = the bits of u),
// the warp table [fs (2n) | hs (5) | gs (K) | es (1) | pad], stride reals a
// unit, with the definitions the gather uses when it builds them itself:
//   fs_j = h+_j + sum_{i outer} rho_ji m_i,   hs_l = sum_{j outer} zz_lj m_j,
//   gs_c = sum_{i outer} zz_{5+c, i} m_i,
//   es = sum_{i outer} (m_i (hz_i + sum_{j > i outer} zz_ij m_j) + iondiag_i(b_i)),
// evaluated in FP64 from the FP64 coupling tables, one thread per unit.
template <typename real>
__global__ void vm_unit_tables_kernel(const double* __restrict__ t, const TabLayout L, int n, int K, long long nunits,
                                      int stride, real* __restrict__ out) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nunits) return;
  const int lo = kLaneBits + K;
  const unsigned long long base = (unsigned long long)u << lo;
  auto m = [&](int i) { return ((base >> i) & 1ull) ? 0.5 : -0.5; };
  auto zz = [&](int i, int j) { return i < j ? t[L.off_zz + i * n + j] : t[L.off_zz + j * n + i]; };
  real* o = out + (size_t)u * stride;
  for (int j = 0; j < n; ++j) {
    double fr = t[L.off_hp + 2 * j], fi = t[L.off_hp + 2 * j + 1];
    for (int i = lo; i < n; ++i) {
      fr += t[L.off_rho + 2 * (j * n + i)] * m(i);
      fi += t[L.off_rho + 2 * (j * n + i) + 1] * m(i);
    }
    o[2 * j] = (real)fr;
    o[2 * j + 1] = (real)fi;
  }
  for (int l = 0; l < kLaneBits; ++l) {
    double h = 0.0;
    for (int j = lo; j < n; ++j) h += zz(l, j) * m(j);
    o[2 * n + l] = (real)h;
  }
  for (int c = 0; c < K; ++c) {
    double g = 0.0;
    for (int i = lo; i < n; ++i) g += zz(kLaneBits + c, i) * m(i);
    o[2 * n + kLaneBits + c] = (real)g;
  }
  double e = 0.0;
  for (int i = lo; i < n; ++i) {
    double zs = t[L.off_hz + i];
    for (int j = i + 1; j < n; ++j) zs += zz(i, j) * m(j);
    e += m(i) * zs + t[L.off_iondiag + i * L.qmax + (int)((base >> i) & 1ull)];
  }
  o[2 * n + kLaneBits + K] = (real)e;
  for (int k = 2 * n + kLaneBits + K + 1; k < stride; ++k) o[k] = (real)0;
}

int vm_unit_table_stride(int n, int K) { return (2 * n + kLaneBits + K + 1 + 1) & ~1; }

int launch_vm_unit_tables(const double* tab_d, const TabLayout& L, int n, int K, long long nunits, void* out, int c64,
                          void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int stride = vm_unit_table_stride(n, K);
  const unsigned grid = (unsigned)((nunits + 127) / 128);
  if (c64) vm_unit_tables_kernel<float><<<grid, 128, 0, st>>>(tab_d, L, n, K, nunits, stride, (float*)out);
  else vm_unit_tables_kernel<double><<<grid, 128, 0, st>>>(tab_d, L, n, K, nunits, stride, (double*)out);
  return (int)cudaGetLastError();
}

// y = c (u.S) x on the vector-major block of a spin-1/2 system (R one-vector
// instances, tiles as in vm_stream_kernel), c = sigma_0 with a.use_sigma0
// (the start block's observable vector) or 1.  With every s_i = 1/2 a row's
// digits are its bits: (u.S x)[mu] = u_z (sum_i m_i) x[mu] + sum_i
// (bit i ? a <1|s+|0> x[mu - 2^i] : conj(a) <0|s-|1> x[mu + 2^i]),
// a = (u_x - i u_y)/2, the terms and coefficients of the general row form.
template <typename real>
__global__ void __launch_bounds__(256) vm_sdir_kernel(const __grid_constant__ LaunchArgs a) {
  using v2 = typename Cx<real>::v2;
  __shared__ InstDesc d;
  __shared__ __align__(16) real site[kMaxSites][4];  // m(down), m(up), <1|s+|0>, <0|s-|1>
  const int bd = blockDim.x;
  int cur = -1;
  real c = 1;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int inst = tile / a.tiles_per_vg;
    if (inst != cur) {
      __syncthreads();
      if (threadIdx.x == 0) d = a.inst[inst];
      __syncthreads();
      if (cur < 0) {  // the system's tables (every instance is a vector of the same system)
        const real* t = reinterpret_cast<const real*>(d.tab);
        for (int i = threadIdx.x; i < d.n; i += bd) {
          site[i][0] = t[d.lay.off_m + i * d.lay.qmax];
          site[i][1] = t[d.lay.off_m + i * d.lay.qmax + 1];
          site[i][2] = t[d.lay.off_up1 + i * d.lay.qmax + 1];
          site[i][3] = t[d.lay.off_dn1 + i * d.lay.qmax];
        }
        __syncthreads();
      }
      c = a.use_sigma0 ? (real)d.sc.sigma[0] : (real)1;
      cur = inst;
    }
    const int n = d.n;
    const real uz = (real)d.obs[0], aur = (real)d.obs[1], aui = (real)d.obs[2];
    const v2* x = reinterpret_cast<const v2*>(d.x);
    v2* y = reinterpret_cast<v2*>(d.y);
    const long long e0 = (long long)(tile - inst * a.tiles_per_vg) * a.rows_per_tile;
    const long long e1 = min(e0 + (long long)a.rows_per_tile, d.dim);
    for (long long mu = e0 + threadIdx.x; mu < e1; mu += bd) {
      real ar = 0, ai = 0, msum = 0;
#pragma unroll 4
      for (int i = 0; i < n; ++i) {  // (unrolled: several sites' gathered loads in flight)
        const typename Cx<real>::v2 mm = *reinterpret_cast<const v2*>(&site[i][0]);
        const typename Cx<real>::v2 cc = *reinterpret_cast<const v2*>(&site[i][2]);
        const bool up = (mu >> i) & 1;
        msum += up ? mm.y : mm.x;
        const v2 xv = __ldg(x + (up ? mu - (1ll << i) : mu + (1ll << i)));
        const real e = up ? cc.x : cc.y;
        const real cr = aur * e, ci = up ? aui * e : -aui * e;
        ar = fma(cr, xv.x, fma(-ci, xv.y, ar));
        ai = fma(cr, xv.y, fma(ci, xv.x, ai));
      }
      const v2 xo = __ldg(x + mu);
      const real dz = uz * msum;
      v2 o;
      o.x = c * fma(dz, xo.x, ar);
      o.y = c * fma(dz, xo.y, ai);
      y[mu] = o;
    }
  }
}

int launch_vm_stream(const LaunchArgs& a, int c64, int grid, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.inline_one || (a.rows_per_tile & 1)) return (int)cudaErrorInvalidValue;
  if (a.mode == kModeStep) {
    if (c64) vm_stream_kernel<float, kModeStep><<<grid, 256, 0, st>>>(a);
    else vm_stream_kernel<double, kModeStep><<<grid, 256, 0, st>>>(a);
  } else if (a.mode == kModeUpdate) {
    if (c64) vm_stream_kernel<float, kModeUpdate><<<grid, 256, 0, st>>>(a);
    else vm_stream_kernel<double, kModeUpdate><<<grid, 256, 0, st>>>(a);
  } else if (a.mode == kModeStartNorm) {
    if (c64) vm_stream_kernel<float, kModeStartNorm><<<grid, 256, 0, st>>>(a);
    else vm_stream_kernel<double, kModeStartNorm><<<grid, 256, 0, st>>>(a);
  } else if (a.mode == kModeApplyS) {
    if (a.max_n > kMaxSites) return (int)cudaErrorInvalidValue;
    if (c64) vm_sdir_kernel<float><<<grid, 256, 0, st>>>(a);
    else vm_sdir_kernel<double><<<grid, 256, 0, st>>>(a);
  } else {
    return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <typename real, int K, bool MP>
static const void* vm_fn(int minb) {
  if (minb == 1) return (const void*)vm_kernel<real, K, MP, 1>;
  if (!MP && minb > 2) return (const void*)vm_kernel<real, K, false, 3>;
  return (const void*)vm_kernel<real, K, MP, 2>;
}

template <typename real, int K>
static int launch_vm_k(const LaunchArgs& a, int minb, int grid, int threads, size_t smem, cudaStream_t st) {
  if ((minb == 1) != (threads == 512)) return (int)cudaErrorInvalidValue;
  if (!a.single_pass) {
    if (minb == 1) vm_kernel<real, K, true, 1><<<grid, threads, smem, st>>>(a);
    else vm_kernel<real, K, true, 2><<<grid, threads, smem, st>>>(a);
  } else if (minb == 1) {
    vm_kernel<real, K, false, 1><<<grid, threads, smem, st>>>(a);
  } else if (minb > 2) {
    vm_kernel<real, K, false, 3><<<grid, threads, smem, st>>>(a);
  } else {
    vm_kernel<real, K, false, 2><<<grid, threads, smem, st>>>(a);
  }
  return (int)cudaGetLastError();
}

int launch_vm(const LaunchArgs& a, int K, int minb, int c64, int grid, int threads, size_t smem, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.mode != kModeApply) return (int)cudaErrorInvalidValue;
  if (c64) {
    if (K == 3) return launch_vm_k<float, 3>(a, minb, grid, threads, smem, st);
    if (K == 4) return launch_vm_k<float, 4>(a, minb, grid, threads, smem, st);
  } else {
    if (K == 3) return launch_vm_k<double, 3>(a, minb, grid, threads, smem, st);
    if (K == 4) return launch_vm_k<double, 4>(a, minb, grid, threads, smem, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <typename real, int K>
static void vm_variants(std::vector<const void*>& ks) {
  for (int minb : {1, 2, 3}) {
    ks.push_back(vm_fn<real, K, false>(minb));
    ks.push_back(vm_fn<real, K, true>(minb));
  }
}

int prepare_vm_kernels(size_t smem) {
  std::vector<const void*> ks;
  vm_variants<float, 3>(ks);
  vm_variants<float, 4>(ks);
  vm_variants<double, 3>(ks);
  vm_variants<double, 4>(ks);
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

// Shared-memory carveout (percent of the SM's L1/shared capacity) for the
// launch about to run: what `ctas` resident CTAs of `smem` bytes need, so that
// the remainder stays L1 cache.
int set_vm_carveout(int K, int c64, bool multipass, int min_blocks, size_t smem, int ctas) {
  const void* k = nullptr;
  if (c64) {
    if (K == 3) k = multipass ? vm_fn<float, 3, true>(min_blocks) : vm_fn<float, 3, false>(min_blocks);
    if (K == 4) k = multipass ? vm_fn<float, 4, true>(min_blocks) : vm_fn<float, 4, false>(min_blocks);
  } else {
    if (K == 3) k = multipass ? vm_fn<double, 3, true>(min_blocks) : vm_fn<double, 3, false>(min_blocks);
    if (K == 4) k = multipass ? vm_fn<double, 4, true>(min_blocks) : vm_fn<double, 4, false>(min_blocks);
  }
  if (!k) return (int)cudaErrorInvalidValue;
  const double total = 228.0 * 1024.0;  // shared memory per SM
  const double need = (double)ctas * ((double)smem + 1024.0 + 2048.0);  // + per-CTA reserve and static tables
  const int pct = std::min(100, std::max(1, (int)std::ceil(100.0 * need / total)));
  return (int)cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <typename real, int K>
static cudaError_t vm_occ(int* nb, int minb, bool multipass, int threads, size_t smem) {
  const void* k = multipass ? vm_fn<real, K, true>(minb) : vm_fn<real, K, false>(minb);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k, threads, smem);
}

int vm_max_ctas_per_sm(int K, int minb, int c64, int threads, size_t smem, bool multipass) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (c64) {
    if (K == 3) e = vm_occ<float, 3>(&nb, minb, multipass, threads, smem);
    if (K == 4) e = vm_occ<float, 4>(&nb, minb, multipass, threads, smem);
  } else {
    if (K == 3) e = vm_occ<double, 3>(&nb, minb, multipass, threads, smem);
    if (K == 4) e = vm_occ<double, 4>(&nb, minb, multipass, threads, smem);
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace ftlm
