// CUDA kernels of the FTLM hot path (arxiv 2607.25585, Secs. II.A-II.C):
//  * the matrix-free row-gather H.v over the (2s+1)^N product basis, with
//    the coupling tables of Eq. (3) staged in shared memory and every matrix
//    element evaluated on the fly (no stored matrix, no atomics);
//  * the Lanczos step epilogue fused into the matvec (w = H v_j - beta_j
//    v_{j-1}, in place over v_{j-1}, with the partial sums of
//    alpha_j = Re<v_j|w> and p_j = <v_j|u>), the orthogonalisation update,
//    the start-vector norm and the observable u.S;
//  * deterministic two-stage reductions: per-CTA partials in FP64, then the
//    last CTA to finish sums them in a fixed order and writes the Lanczos
//    scalars (alpha, p, beta, the breakdown test and the vector scales).
//
// Vector blocks are [dim][R] complex, R fastest.  A thread owns one row and
// a chunk of V consecutive vectors (16 bytes: V = 2 for complex64, 1 for
// complex128), so a warp reads whole 512-byte rows when R = 64.
// Lanczos vectors are kept unnormalised: v_j = sigma_j q_j, with sigma_j in
// device memory, which saves a normalisation pass per step.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "ftlm_internal.h"
#include "rows_common.cuh"

namespace ftlm {

// one row of H x; also returns the row's own x values (the Lanczos epilogue uses them)
template <typename real, int V>
__device__ __forceinline__ void h_row(const SmemView& s, const TabLayout& L, int n, long long mu, bool idx32,
                                      const void* __restrict__ x, int R, int col, real* ar, real* ai, real* xr_own,
                                      real* xi_own) {
  GatherSink<real, V> g{x, mu, R, col, ar, ai, xr_own, xi_own};
  row_terms<real>(s, L, n, mu, idx32, g);
}

// one row of (u.S) x: u_z sum_i m_i x_mu + a_u <a|s+|a-1> x_{mu - s_i} + conj(a_u) <a|s-|a+1> x_{mu + s_i}
template <typename real, int V>
__device__ __forceinline__ void s_row(const SmemView& s, const TabLayout& L, int n, long long mu, bool idx32,
                                      const void* __restrict__ x, int R, int col, real uz, real aur, real aui,
                                      real* ar, real* ai) {
  const real* t = reinterpret_cast<const real*>(s.tab);
  const int qm = L.qmax;
  real msum = 0;
#pragma unroll
  for (int v = 0; v < V; ++v) ar[v] = ai[v] = 0;
  unsigned long long rem = (unsigned long long)mu;
  unsigned rem32 = (unsigned)mu;
  for (int i = 0; i < n; ++i) {
    int a_i;
    if (idx32) {
      const unsigned nq = rem32 / (unsigned)s.q[i];
      a_i = (int)(rem32 - nq * (unsigned)s.q[i]);
      rem32 = nq;
    } else {
      const unsigned long long nq = rem / (unsigned long long)s.q[i];
      a_i = (int)(rem - nq * (unsigned long long)s.q[i]);
      rem = nq;
    }
    msum += t[L.off_m + i * qm + a_i];
    if (a_i >= 1) {
      const real e = t[L.off_up1 + i * qm + a_i];
      gather_mac<real, V>(x, mu - s.stride[i], R, col, aur * e, aui * e, ar, ai);
    }
    if (a_i + 1 < s.q[i]) {
      const real e = t[L.off_dn1 + i * qm + a_i];
      gather_mac<real, V>(x, mu + s.stride[i], R, col, aur * e, -aui * e, ar, ai);
    }
  }
  real xr[V], xi[V];
  VecIO<real, V>::ldg(x, mu * R + col, xr, xi);
  const real dz = uz * msum;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    ar[v] = fma(dz, xr[v], ar[v]);
    ai[v] = fma(dz, xi[v], ai[v]);
  }
}

// ---------------------------------------------------------------------------
// fixed-order reductions
// ---------------------------------------------------------------------------
// Sums thread accumulators acc[V*kNumPartials] over the threads of the CTA
// that own the same vector chunk (tid % C) and writes the CTA's partials for
// instance `inst`.  All threads must call it.
template <int V>
__device__ void flush_partials(const LaunchArgs& a, const SmemView& s, int inst, double* acc) {
  const int np = V * kNumPartials;
  const int C = a.C;
  if (C <= 32 && (32 % C) == 0) {
    // the threads of one chunk (tid % C) within a warp are lanes chunk, chunk + C, ...:
    // add them by shuffles, then the warps' sums in warp order (fixed, deterministic)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < np; ++k) {
      double v = acc[k];
      for (int o = 16; o >= C; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[k] = v;
    }
    __syncthreads();
    if (lane < C)
      for (int k = 0; k < np; ++k) s.red[(warp * C + lane) * np + k] = acc[k];
    __syncthreads();
    if ((int)threadIdx.x < C) {
      double* out = a.partials + ((size_t)inst * gridDim.x + blockIdx.x) * (size_t)a.R * kNumPartials;
      for (int k = 0; k < np; ++k) {
        double sum = 0.0;
        for (int w = 0; w < nw; ++w) sum += s.red[(w * C + threadIdx.x) * np + k];
        const int v = k / kNumPartials, c = k % kNumPartials;
        out[(threadIdx.x * V + v) * kNumPartials + c] = sum;
      }
    }
    __syncthreads();
    for (int k = 0; k < np; ++k) acc[k] = 0.0;
    return;
  }
  __syncthreads();
  for (int k = 0; k < np; ++k) s.red[threadIdx.x * np + k] = acc[k];
  __syncthreads();
  const int per = blockDim.x / C;
  if ((int)threadIdx.x < C) {
    double sum[V * kNumPartials];
    for (int k = 0; k < np; ++k) sum[k] = 0.0;
    for (int r = 0; r < per; ++r)
      for (int k = 0; k < np; ++k) sum[k] += s.red[(threadIdx.x + r * C) * np + k];
    double* out = a.partials + ((size_t)inst * gridDim.x + blockIdx.x) * (size_t)a.R * kNumPartials;
    for (int v = 0; v < V; ++v)
      for (int c = 0; c < kNumPartials; ++c) out[(threadIdx.x * V + v) * kNumPartials + c] = sum[v * kNumPartials + c];
  }
  __syncthreads();
  for (int k = 0; k < np; ++k) acc[k] = 0.0;
}

// ---------------------------------------------------------------------------
// the tile loop shared by every mode
// ---------------------------------------------------------------------------
template <typename real, int V, int MODE>
// complex64: three 256-thread CTAs per SM (at most 85 registers a thread)
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 3 : 1) rows_kernel(const __grid_constant__ LaunchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kPartials = MODE == kModeLanczos || MODE == kModeEpilogue || MODE == kModeUpdate ||
                             MODE == kModeStartNorm || MODE == kModeStep;
  const SmemView s = carve<real>(smem_raw, a, kPartials ? V : 0);  // no reduction space without partial sums
  __shared__ InstDesc d;
  __shared__ int is_last;
  const InstDesc* insts = a.inline_one ? &a.one : a.inst;
  constexpr int NP = V * kNumPartials;
  double acc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = 0.0;

  const int C = a.C;
  const int chunk = threadIdx.x % C;   // fixed per thread: blockDim is a multiple of C
  const int col = chunk * V;

  if (kPartials) {  // zero this CTA's slots of every instance
    for (int inst = 0; inst < a.n_inst; ++inst) {
      double* out = a.partials + ((size_t)inst * gridDim.x + blockIdx.x) * (size_t)a.R * kNumPartials;
      for (int k = threadIdx.x; k < a.R * kNumPartials; k += blockDim.x) out[k] = 0.0;
    }
  }
  int cur = -1;
  real sig[V], bsp[V], coef[V];  // per-vector scalars of the current instance
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int inst = a.inline_one ? 0 : find_instance(a.tile_start, a.n_inst, tile);
    if (inst != cur) {
      if (kPartials && cur >= 0) flush_partials<V>(a, s, cur, acc);
      __syncthreads();
      if (threadIdx.x == 0) d = insts[inst];
      __syncthreads();
      if (MODE == kModeApply || MODE == kModeLanczos || MODE == kModeApplyS) stage_instance<real>(d, s);
      const int j = a.step;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int k = min(col + v, a.R - 1);
        sig[v] = bsp[v] = coef[v] = 0;
        if (MODE == kModeLanczos || MODE == kModeEpilogue || MODE == kModeStep) {
          sig[v] = (real)d.sc.sigma[(size_t)j * d.sc.ss + k];
          if (!a.first) bsp[v] = (real)(d.sc.beta[(size_t)(j - 1) * d.sc.ss + k] * d.sc.sigma[(size_t)(j - 1) * d.sc.ss + k]);
          if (MODE == kModeStep)
            coef[v] = (real)(d.sc.alpha[(size_t)j * d.sc.ss + k] * d.sc.sigma[(size_t)j * d.sc.ss + k]);
        } else if (MODE == kModeUpdate) {
          coef[v] = a.update_no_alpha ? (real)0
                                      : (real)(d.sc.alpha[(size_t)j * d.sc.ss + k] * d.sc.sigma[(size_t)j * d.sc.ss + k]);
        } else if (MODE == kModeApplyS) {
          coef[v] = a.use_sigma0 ? (real)d.sc.sigma[k] : (real)1;
        } else if (MODE == kModeScale) {
          coef[v] = (real)d.sc.sigma[k];
        }
      }
      cur = inst;
      __syncthreads();
    }
    const int first_tile = a.inline_one ? 0 : __ldg(a.tile_start + inst);
    const long long row0 = (long long)(tile - first_tile) * a.rows_per_tile;
    const bool idx32 = d.dim <= 0xffffffffll;
    real pacc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) pacc[k] = 0;
    constexpr bool kElementwise = MODE == kModeEpilogue || MODE == kModeUpdate || MODE == kModeStartNorm ||
                                  MODE == kModeScale || MODE == kModeStep;
    if (kElementwise) {
      // element e = row * R + col: linear over the tile; blockDim * V is a
      // multiple of R, so each thread keeps its vector chunk
      const long long e_end = min(row0 + a.rows_per_tile, d.dim) * a.R;
      const long long step = (long long)blockDim.x * V;
      long long e = row0 * a.R + (long long)threadIdx.x * V;
      // loads of several groups in flight per thread before their stores (the
      // compiler cannot move a group's loads above the previous group's stores)
      constexpr int kU = V >= 4 ? 1 : 4 / V;
      if (MODE == kModeStep) {
        step_stream<real, V, 4>(d, a, e, e_end, step, sig, bsp, coef, pacc);
      } else if (MODE == kModeUpdate) {
        update_stream<real, V, kU>(d, e, e_end, step, coef, pacc);
      } else if (MODE == kModeEpilogue) {
        epilogue_stream<real, V, kU>(d, a, e, e_end, step, sig, bsp, pacc);
      } else {
        for (; e + step < e_end; e += 2 * step) {
          elementwise_item<real, V, MODE>(d, a, e, sig, bsp, coef, pacc);
          elementwise_item<real, V, MODE>(d, a, e + step, sig, bsp, coef, pacc);
        }
        if (e < e_end) elementwise_item<real, V, MODE>(d, a, e, sig, bsp, coef, pacc);
      }
    } else {
    const int items = a.rows_per_tile * C;
    for (int item = threadIdx.x; item < items; item += blockDim.x) {
      const long long row = row0 + item / C;
      if (row >= d.dim) break;
      const long long idx = row * a.R + col;
      if (MODE == kModeApply || MODE == kModeLanczos || MODE == kModeEpilogue) {
        real ar[V], ai[V], xr[V], xi[V];
        if (MODE == kModeEpilogue) {  // H q_j from the gather launch, own row of q_j
          VecIO<real, V>::ldg(d.hq, idx, ar, ai);
          VecIO<real, V>::ldg(d.x, idx, xr, xi);
        } else {
          h_row<real, V>(s, d.lay, d.n, row, idx32, d.x, a.R, col, ar, ai, xr, xi);
        }
        if (MODE == kModeApply) {
          VecIO<real, V>::st(d.y, idx, ar, ai);
        } else {
          real wr[V], wi[V];
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
          real ur[V], ui[V];
          VecIO<real, V>::ldg(d.u, idx, ur, ui);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const real vr = sig[v] * xr[v], vi = sig[v] * xi[v];
            pacc[v * kNumPartials + 0] += vr * wr[v] + vi * wi[v];     // Re <v|w>
            pacc[v * kNumPartials + 1] += vr * ur[v] + vi * ui[v];     // Re <v|u>
            pacc[v * kNumPartials + 2] += vr * ui[v] - vi * ur[v];     // Im <v|u>
          }
        }
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
      } else if (MODE == kModeApplyS) {
        real ar[V], ai[V];
        s_row<real, V>(s, d.lay, d.n, row, idx32, d.x, a.R, col, (real)d.obs[0], (real)d.obs[1], (real)d.obs[2],
                       ar, ai);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          ar[v] *= coef[v];
          ai[v] *= coef[v];
        }
        VecIO<real, V>::st(d.y, idx, ar, ai);
      }
    }
    }
    if (kPartials) {
#pragma unroll
      for (int k = 0; k < NP; ++k) acc[k] += (double)pacc[k];
    }
  }
  if (!kPartials) return;
  if (cur >= 0) flush_partials<V>(a, s, cur, acc);
  // last CTA to arrive reduces every CTA's partials in a fixed order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize(a, insts);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// ---------------------------------------------------------------------------
// the vector-major general H.v
// ---------------------------------------------------------------------------
// The gather of row_terms against V vectors of one system that lie dim
// elements apart (each vector contiguous): a warp's 32 lanes own 32
// consecutive rows, so every load of a term is 32 consecutive values of one
// vector (one 256-byte line pair), and the row's matrix elements are formed
// once for its V vectors.
template <typename real, int V>
struct VmGatherSink {
  using v2 = typename Cx<real>::v2;
  const v2* x;    // vector 0 of the group
  long long mu;   // the row
  long long vs;   // elements from one vector of the group to the next
  real *ar, *ai;
  __device__ __forceinline__ void diag(real dv) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const v2 xv = __ldg(x + v * vs + mu);
      ar[v] = dv * xv.x;
      ai[v] = dv * xv.y;
    }
  }
  __device__ __forceinline__ void term(long long nu, real cr, real ci) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const v2 xv = __ldg(x + v * vs + nu);
      ar[v] = fma(cr, xv.x, ar[v]);
      ar[v] = fma(-ci, xv.y, ar[v]);
      ai[v] = fma(cr, xv.y, ai[v]);
      ai[v] = fma(ci, xv.x, ai[v]);
    }
  }
};

// y = H x on vector-major blocks.  a.inst holds one descriptor per vector
// (one-vector instances, the V vectors of a group consecutive and dim apart);
// a.tile_start is the prefix sum of tiles over the groups (a.n_inst groups),
// a tile being a.rows_per_tile rows of one group.  Tiles go round-robin over
// the CTAs, so CTAs running together share a group's neighbourhood in L2.
template <typename real, int V>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 3 : 2) rows_vm_kernel(const __grid_constant__ LaunchArgs a) {
  using v2 = typename Cx<real>::v2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmemView s = carve<real>(smem_raw, a, 0);
  __shared__ InstDesc d;
  const InstDesc* insts = a.inline_one ? &a.one : a.inst;
  int cur = -1;
  const void* staged = nullptr;  // tables of the system now in shared memory
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int g = a.inline_one ? 0 : find_instance(a.tile_start, a.n_inst, tile);
    if (g != cur) {
      __syncthreads();
      if (threadIdx.x == 0) d = insts[(size_t)g * V];
      __syncthreads();
      if (d.tab != staged) {  // the groups of one system share its tables
        stage_instance<real>(d, s);
        staged = d.tab;
      }
      cur = g;
      __syncthreads();
    }
    const int first_tile = a.inline_one ? 0 : __ldg(a.tile_start + g);
    const long long row0 = (long long)(tile - first_tile) * a.rows_per_tile;
    const long long row_end = min(row0 + a.rows_per_tile, d.dim);
    const bool idx32 = d.dim <= 0xffffffffll;
    const v2* x = reinterpret_cast<const v2*>(d.x);
    v2* y = reinterpret_cast<v2*>(d.y);
    for (long long mu = row0 + threadIdx.x; mu < row_end; mu += blockDim.x) {
      real ar[V], ai[V];
      VmGatherSink<real, V> sink{x, mu, d.dim, ar, ai};
      row_terms<real>(s, d.lay, d.n, mu, idx32, sink);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        v2 o;
        o.x = ar[v];
        o.y = ai[v];
        y[v * d.dim + mu] = o;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// start vectors: Philox4x32-10 (Salmon et al., SC'11), Box-Muller in FP64
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(unsigned& c0, unsigned& c1, unsigned& c2, unsigned& c3, unsigned k0,
                                             unsigned k1) {
  const unsigned lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
  const unsigned lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
  const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

__device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c[0], c[1], c[2], c[3], k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ double unit53(unsigned hi, unsigned lo) {
  const unsigned long long k = ((unsigned long long)hi << 21) | ((unsigned long long)lo >> 11);
  return ((double)k + 1.0) * (1.0 / 9007199254740992.0);
}

// VMAJ: vector-major output (element e = k * dim + nu), else row-major (e = nu * R + k).
template <typename real, bool VMAJ>
__global__ void start_random_kernel(long long dim, int R, unsigned long long seed, unsigned long long vec_offset,
                                    real* out) {
  const long long total = dim * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nu = VMAJ ? e % dim : e / R;
    const unsigned long long rg = vec_offset + (unsigned long long)(VMAJ ? e / dim : e - nu * R);
    unsigned c[4] = {(unsigned)nu, (unsigned)((unsigned long long)nu >> 32), (unsigned)rg, (unsigned)(rg >> 32)};
    philox4x32_10(c, (unsigned)seed, (unsigned)(seed >> 32));
    const double u1 = unit53(c[0], c[1]);
    const double u2 = unit53(c[2], c[3]);
    const double rho = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[2 * e] = (real)(rho * cs);
    out[2 * e + 1] = (real)(rho * sn);
  }
}

template <typename real, bool VMAJ>
__global__ void start_basis_kernel(long long dim, int R, unsigned long long basis_offset, real* out) {
  const long long total = dim * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nu = VMAJ ? e % dim : e / R;
    const long long k = VMAJ ? e / dim : e - nu * R;
    out[2 * e] = (real)((unsigned long long)nu == basis_offset + (unsigned long long)k ? 1.0 : 0.0);
    out[2 * e + 1] = (real)0;
  }
}

// Parity of the digit sum sum_i a_i(nu) (a_i = m_i + s_i): the sign of the
// time-reversed basis state, (-1)^(sum_i (s_i - m_i)) at the image (Sec. II.B).
__device__ __forceinline__ int digit_parity(long long nu, int n, const int* q, int all_half) {
  if (all_half) return __popcll((unsigned long long)nu) & 1;
  int sum = 0;
  for (int i = 0; i < n; ++i) {
    const int qi = __ldg(q + i);
    sum += (int)(nu % qi);
    nu /= qi;
  }
  return sum & 1;
}

// Pairs of mutually time-reversed random vectors (Sec. II.B, tau = 1 in
// Sec. III): global vector v = vec_offset + k is random vector v / 2 of the
// Philox stream when v is even and its time reverse when v is odd,
//   (Theta r)[nu] = (-1)^(sum_i a_i(nu)) conj(r[d - 1 - nu]),
// since Theta = exp(-i pi S^y) K maps every digit a_i to 2 s_i - a_i, i.e.
// the index nu to d - 1 - nu.  Unnormalised, like start_random_kernel.
template <typename real, bool VMAJ>
__global__ void start_pairs_kernel(long long dim, int R, unsigned long long seed, unsigned long long vec_offset,
                                   int n, const int* q, int all_half, real* out) {
  const long long total = dim * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nu = VMAJ ? e % dim : e / R;
    const unsigned long long v = vec_offset + (unsigned long long)(VMAJ ? e / dim : e - nu * R);
    const bool rev = (v & 1ull) != 0;
    const long long src = rev ? dim - 1 - nu : nu;
    const unsigned long long rg = v >> 1;
    unsigned c[4] = {(unsigned)src, (unsigned)((unsigned long long)src >> 32), (unsigned)rg, (unsigned)(rg >> 32)};
    philox4x32_10(c, (unsigned)seed, (unsigned)(seed >> 32));
    const double u1 = unit53(c[0], c[1]);
    const double u2 = unit53(c[2], c[3]);
    const double rho = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    double re = rho * cs, im = rho * sn;
    if (rev) {
      im = -im;
      if (digit_parity(nu, n, q, all_half)) {
        re = -re;
        im = -im;
      }
    }
    out[2 * e] = (real)re;
    out[2 * e + 1] = (real)im;
  }
}

// y = Theta x on a row-major [d][R] block: y[nu][k] = (-1)^(sum a_i(nu)) conj(x[d-1-nu][k]).
// V consecutive vectors of a row per thread (16-byte accesses for complex64
// with even R), two items per loop trip.
template <typename real, int V>
__global__ void time_reverse_kernel(long long dim, int R, int n, const int* q, int all_half, const real* x,
                                    real* y) {
  const long long items = dim * R / V;
  const int C = R / V;  // items per row
  auto one = [&](long long it) {
    const long long nu = it / C;
    const long long idx = it * V;               // complex index of the first value
    const long long src = (dim - 1 - nu) * R + (idx - nu * R);
    real re[V], im[V];
    VecIO<real, V>::ldg(x, src, re, im);
    const real sg = digit_parity(nu, n, q, all_half) ? (real)-1 : (real)1;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      re[v] *= sg;
      im[v] *= -sg;
    }
    VecIO<real, V>::st(y, idx, re, im);
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; it + stride < items; it += 2 * stride) {
    one(it);
    one(it + stride);
  }
  if (it < items) one(it);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t rows_smem_bytes(const LaunchArgs& a, int c64, int threads, int Vmax) {
  const int V = Vmax > 0 ? Vmax : (c64 ? 2 : 1);
  const size_t realsz = c64 ? 4 : 8;
  size_t off = ((size_t)a.tab_reals * realsz + 15) & ~size_t(15);
  off += (size_t)a.max_n * 8;
  off += ((size_t)a.max_n * 4 + 15) & ~size_t(15);
  off += (size_t)threads * kNumPartials * V * 8;
  off += ((size_t)a.max_n * threads * realsz + 15) & ~size_t(15);  // the per-thread m columns
  off += (size_t)a.max_n * threads;
  return off;
}

// The general gathers that carve no reduction space (rows_vm_kernel,
// cube_gather_kernel): tables, strides, radices, per-thread m and digit columns.
size_t gather_smem_bytes(const LaunchArgs& a, int c64, int threads) {
  const size_t realsz = c64 ? 4 : 8;
  size_t off = ((size_t)a.tab_reals * realsz + 15) & ~size_t(15);
  off += (size_t)a.max_n * 8;
  off += ((size_t)a.max_n * 4 + 15) & ~size_t(15);
  off += ((size_t)a.max_n * threads * realsz + 15) & ~size_t(15);
  off += (size_t)a.max_n * threads;
  return off;
}

template <typename real, int V, int MODE>
static int launch_one(const LaunchArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  rows_kernel<real, V, MODE><<<grid, threads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename real, int V>
static int allow_smem(int bytes) {
  const void* ks[] = {(const void*)rows_kernel<real, V, kModeApply>, (const void*)rows_kernel<real, V, kModeLanczos>,
                      (const void*)rows_kernel<real, V, kModeUpdate>, (const void*)rows_kernel<real, V, kModeStartNorm>,
                      (const void*)rows_kernel<real, V, kModeApplyS>, (const void*)rows_kernel<real, V, kModeScale>,
                      (const void*)rows_kernel<real, V, kModeEpilogue>, (const void*)rows_kernel<real, V, kModeStep>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

// Raises the dynamic shared-memory limit of every row kernel; called outside
// stream capture before the first launch that needs more than 48 KB.
int prepare_rows_kernels(size_t smem) {
  int e = allow_smem<float, 2>((int)smem);
  if (!e) e = allow_smem<float, 1>((int)smem);
  if (!e) e = allow_smem<double, 1>((int)smem);
  const void* wide[] = {(const void*)rows_kernel<float, 4, kModeApply>, (const void*)rows_kernel<float, 8, kModeApply>};
  for (const void* k : wide)
    if (!e) e = (int)cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

// H.v with V = 4 or 8 complex64 vectors per thread (a.C = R / V): the row's
// matrix elements are computed once for V vectors (16 per thread, one thread
// per row at R = 16, was twice as slow: the loads no longer coalesce).
int launch_rows_wide(const LaunchArgs& a, int V, int grid, int threads, size_t smem, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.mode != kModeApply || a.R % V != 0 || a.C != a.R / V) return (int)cudaErrorInvalidValue;
  if (V == 8) rows_kernel<float, 8, kModeApply><<<grid, threads, smem, st>>>(a);
  else if (V == 4) rows_kernel<float, 4, kModeApply><<<grid, threads, smem, st>>>(a);
  else return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

template <typename real, int V>
static int launch_mode(const LaunchArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  switch (a.mode) {
    case kModeApply: return launch_one<real, V, kModeApply>(a, grid, threads, smem, st);
    case kModeLanczos: return launch_one<real, V, kModeLanczos>(a, grid, threads, smem, st);
    case kModeUpdate: return launch_one<real, V, kModeUpdate>(a, grid, threads, smem, st);
    case kModeStartNorm: return launch_one<real, V, kModeStartNorm>(a, grid, threads, smem, st);
    case kModeApplyS: return launch_one<real, V, kModeApplyS>(a, grid, threads, smem, st);
    case kModeScale: return launch_one<real, V, kModeScale>(a, grid, threads, smem, st);
    case kModeEpilogue: return launch_one<real, V, kModeEpilogue>(a, grid, threads, smem, st);
    case kModeStep: return launch_one<real, V, kModeStep>(a, grid, threads, smem, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_rows(const LaunchArgs& a, int c64, int grid, int threads, size_t smem, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (c64) {
    if (a.R % 2 == 0) return launch_mode<float, 2>(a, grid, threads, smem, st);
    return launch_mode<float, 1>(a, grid, threads, smem, st);
  }
  return launch_mode<double, 1>(a, grid, threads, smem, st);
}

template <typename real, int V>
static const void* rows_vm_fn() {
  return (const void*)rows_vm_kernel<real, V>;
}

static const void* rows_vm_pick(int V, int c64) {
  if (c64) {
    if (V == 8) return rows_vm_fn<float, 8>();
    if (V == 4) return rows_vm_fn<float, 4>();
    if (V == 2) return rows_vm_fn<float, 2>();
    if (V == 1) return rows_vm_fn<float, 1>();
  } else {
    if (V == 4) return rows_vm_fn<double, 4>();
    if (V == 2) return rows_vm_fn<double, 2>();
    if (V == 1) return rows_vm_fn<double, 1>();
  }
  return nullptr;
}

int rows_vm_supported(int V, int c64) { return rows_vm_pick(V, c64) != nullptr; }

int prepare_rows_vm(int V, int c64, size_t smem) {
  const void* k = rows_vm_pick(V, c64);
  if (!k) return (int)cudaErrorInvalidValue;
  return (int)cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int rows_vm_ctas_per_sm(int V, int c64, int threads, size_t smem) {
  const void* k = rows_vm_pick(V, c64);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess || n < 1) return 1;
  return n;
}

int launch_rows_vm(const LaunchArgs& a, int V, int c64, int grid, int threads, size_t smem, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.mode != kModeApply) return (int)cudaErrorInvalidValue;
  if (c64) {
    if (V == 8) rows_vm_kernel<float, 8><<<grid, threads, smem, st>>>(a);
    else if (V == 4) rows_vm_kernel<float, 4><<<grid, threads, smem, st>>>(a);
    else if (V == 2) rows_vm_kernel<float, 2><<<grid, threads, smem, st>>>(a);
    else if (V == 1) rows_vm_kernel<float, 1><<<grid, threads, smem, st>>>(a);
    else return (int)cudaErrorInvalidValue;
  } else {
    if (V == 4) rows_vm_kernel<double, 4><<<grid, threads, smem, st>>>(a);
    else if (V == 2) rows_vm_kernel<double, 2><<<grid, threads, smem, st>>>(a);
    else if (V == 1) rows_vm_kernel<double, 1><<<grid, threads, smem, st>>>(a);
    else return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int rows_max_ctas_per_sm(int c64, int threads, size_t smem, int wideV) {
  int n = 0;
  cudaError_t e;
  // the caller has raised the shared-memory limit to >= smem
  if (wideV == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_kernel<float, 8, kModeApply>, threads, smem);
  else if (wideV == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_kernel<float, 4, kModeApply>, threads, smem);
  else if (c64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_kernel<float, 2, kModeLanczos>, threads, smem);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_kernel<double, 1, kModeLanczos>, threads, smem);
  return (e == cudaSuccess && n > 0) ? n : 1;
}

static int elementwise_grid(long long total) {
  const long long want = (total + 255) / 256;
  return (int)(want < 152LL * 16 ? want : 152LL * 16);
}

int launch_start_random(const InstDesc* inst_host, const InstDesc*, int R, uint64_t seed, uint64_t vec_offset,
                        void* out, int c64, void* stream, int vector_major) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long dim = inst_host->dim;
  const int grid = elementwise_grid(dim * R);
  if (c64) {
    if (vector_major) start_random_kernel<float, true><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, (float*)out);
    else start_random_kernel<float, false><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, (float*)out);
  } else {
    if (vector_major) start_random_kernel<double, true><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, (double*)out);
    else start_random_kernel<double, false><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, (double*)out);
  }
  return (int)cudaGetLastError();
}

int launch_start_basis(long long dim, int R, uint64_t basis_offset, void* out, int c64, void* stream,
                       int vector_major) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = elementwise_grid(dim * R);
  if (c64) {
    if (vector_major) start_basis_kernel<float, true><<<grid, 256, 0, st>>>(dim, R, basis_offset, (float*)out);
    else start_basis_kernel<float, false><<<grid, 256, 0, st>>>(dim, R, basis_offset, (float*)out);
  } else {
    if (vector_major) start_basis_kernel<double, true><<<grid, 256, 0, st>>>(dim, R, basis_offset, (double*)out);
    else start_basis_kernel<double, false><<<grid, 256, 0, st>>>(dim, R, basis_offset, (double*)out);
  }
  return (int)cudaGetLastError();
}

int launch_start_pairs(const InstDesc* h, int R, uint64_t seed, uint64_t vec_offset, void* out, int c64,
                       void* stream, int vector_major) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long dim = h->dim;
  const int grid = elementwise_grid(dim * R);
  if (c64) {
    if (vector_major)
      start_pairs_kernel<float, true><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, h->n, h->q, h->all_half, (float*)out);
    else
      start_pairs_kernel<float, false><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, h->n, h->q, h->all_half, (float*)out);
  } else {
    if (vector_major)
      start_pairs_kernel<double, true><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, h->n, h->q, h->all_half, (double*)out);
    else
      start_pairs_kernel<double, false><<<grid, 256, 0, st>>>(dim, R, seed, vec_offset, h->n, h->q, h->all_half, (double*)out);
  }
  return (int)cudaGetLastError();
}

int launch_time_reverse(const InstDesc* h, const void* x, void* y, int R, int c64, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long dim = h->dim;
  const int grid = elementwise_grid(dim * R);
  if (c64 && R % 2 == 0)
    time_reverse_kernel<float, 2><<<grid, 256, 0, st>>>(dim, R, h->n, h->q, h->all_half, (const float*)x, (float*)y);
  else if (c64)
    time_reverse_kernel<float, 1><<<grid, 256, 0, st>>>(dim, R, h->n, h->q, h->all_half, (const float*)x, (float*)y);
  else
    time_reverse_kernel<double, 1><<<grid, 256, 0, st>>>(dim, R, h->n, h->q, h->all_half, (const double*)x, (double*)y);
  return (int)cudaGetLastError();
}

// dst[k * dim + nu] = src[nu * R + k]: a row-major block to the vector-major
// layout.  Each CTA moves a 32-row x 32-vector tile through shared memory so
// that both the reads and the writes are coalesced.
template <typename v2>
__global__ void to_vector_major_kernel(const v2* __restrict__ src, v2* __restrict__ dst, long long dim, int R) {
  __shared__ v2 tile[32][33];
  const long long row_tiles = (dim + 31) / 32;
  const int vec_tiles = (R + 31) / 32;
  for (long long t = blockIdx.x; t < row_tiles * vec_tiles; t += gridDim.x) {
    const long long nu0 = (t / vec_tiles) * 32;
    const int k0 = (int)(t % vec_tiles) * 32;
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const long long nu = nu0 + i;
      const int k = k0 + threadIdx.x;
      if (nu < dim && k < R) tile[i][threadIdx.x] = src[nu * R + k];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const int k = k0 + i;
      const long long nu = nu0 + threadIdx.x;
      if (nu < dim && k < R) dst[(long long)k * dim + nu] = tile[threadIdx.x][i];
    }
  }
}

int launch_to_vector_major(const void* src, void* dst, long long dim, int R, int c64, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long tiles = ((dim + 31) / 32) * ((R + 31) / 32);
  const int grid = (int)(tiles < 152LL * 16 ? tiles : 152LL * 16);
  const dim3 block(32, 8);
  if (c64) to_vector_major_kernel<float2><<<grid, block, 0, st>>>((const float2*)src, (float2*)dst, dim, R);
  else to_vector_major_kernel<double2><<<grid, block, 0, st>>>((const double2*)src, (double2*)dst, dim, R);
  return (int)cudaGetLastError();
}

// dst[nu * R + k] = src[k * dim + nu]: a vector-major block back to the
// row-major layout, through 32 x 32 shared-memory tiles as above.
template <typename v2>
__global__ void from_vector_major_kernel(const v2* __restrict__ src, v2* __restrict__ dst, long long dim, int R) {
  __shared__ v2 tile[32][33];
  const long long row_tiles = (dim + 31) / 32;
  const int vec_tiles = (R + 31) / 32;
  for (long long t = blockIdx.x; t < row_tiles * vec_tiles; t += gridDim.x) {
    const long long nu0 = (t / vec_tiles) * 32;
    const int k0 = (int)(t % vec_tiles) * 32;
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const int k = k0 + i;
      const long long nu = nu0 + threadIdx.x;
      if (nu < dim && k < R) tile[threadIdx.x][i] = src[(long long)k * dim + nu];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const long long nu = nu0 + i;
      const int k = k0 + threadIdx.x;
      if (nu < dim && k < R) dst[nu * R + k] = tile[i][threadIdx.x];
    }
  }
}

int launch_from_vector_major(const void* src, void* dst, long long dim, int R, int c64, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long tiles = ((dim + 31) / 32) * ((R + 31) / 32);
  const int grid = (int)(tiles < 152LL * 16 ? tiles : 152LL * 16);
  const dim3 block(32, 8);
  if (c64) from_vector_major_kernel<float2><<<grid, block, 0, st>>>((const float2*)src, (float2*)dst, dim, R);
  else from_vector_major_kernel<double2><<<grid, block, 0, st>>>((const double2*)src, (double2*)dst, dim, R);
  return (int)cudaGetLastError();
}

int launch_copy_block(const void* src, void* dst, size_t bytes, void* stream) {
  return (int)cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
}

int device_sm_count() {
  static int cached[64] = {};  // per device ordinal; queried once, outside any stream capture
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

long long device_l2_bytes() {
  static long long cached[64] = {};
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  if (cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

}  // namespace ftlm
