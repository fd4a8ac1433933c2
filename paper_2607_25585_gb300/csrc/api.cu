// C ABI of the FTLM library (include/ftlm.h): system objects, the H.v, u.S
// and start-block entry points, and the FTLM driver (arxiv 2607.25585,
// Eqs. 4-5 and Sec. II.C): start block, M Lanczos steps captured in one CUDA
// graph, then the host eigensolve and Boltzmann sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ftlm_internal.h"

using namespace ftlm;

namespace {

thread_local std::string g_err;

ftlm_status fail(ftlm_status s, const std::string& m) {
  g_err = m;
  return s;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e__ = (call);                                                                     \
    if (e__ != cudaSuccess) {                                                                     \
      cudaGetLastError();                                                                         \
      return fail(e__ == cudaErrorMemoryAllocation ? FTLM_ERR_OUT_OF_MEMORY : FTLM_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e__));                           \
    }                                                                                             \
  } while (0)

#define CKI(expr)                                                                                  \
  do {                                                                                             \
    int e__ = (expr);                                                                              \
    if (e__ != 0) {                                                                                \
      cudaGetLastError();                                                                          \
      return fail(FTLM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString((cudaError_t)e__)); \
    }                                                                                              \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (bytes >= b && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    else p = nullptr;
    return e;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// system object
// ---------------------------------------------------------------------------
struct ftlm_system {
  HostSystem hs;
  int device = 0;
  DevBuf tab_f, tab_d;   // coupling tables, float and double
  DevBuf stride, q;
  cudaStream_t own_stream = nullptr;  // runs capture and launch their graphs here
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // order own_stream after / before the caller's stream
  uint64_t id = 0;       // unique per system
  uint64_t gen = 0;      // bumped whenever the workspace is reallocated
  DevBuf A, B, U, scal;  // Lanczos workspace: two vector blocks, the observable block, scalars
  DevBuf Hq;             // H q_j when the gather and the step epilogue are separate launches
  DevBuf ep, ecnt, esc;  // start-block scratch: partials, arrival counter, scalars
  DevBuf Vs, Wc, Od;     // symmetric runs: stored Lanczos vectors, partial sums of O, O matrices
  DevBuf Ws;             // symmetric runs: u.S of the stored vectors (when it fits)
  DevBuf Gre;            // re-orthogonalised runs: <q_k|w_r> coefficients [R][M] complex
  DevBuf Ta, Tb;         // ftlm_apply_h on spin-1/2 blocks: x and H x in the vector-major layout
  DevBuf ut[2];          // per-unit coefficient tables of the one-pass vector-major gather, [c64]
  int ut_K[2] = {0, 0};  // the cube size each was built for
  cudaEvent_t ev_apply = nullptr;  // recorded after the last use of Ta, Tb
  bool apply_used = false;
  std::mutex mu;
};

namespace {

std::mutex g_mu;
uint64_t g_next_id = 1;
size_t g_prepared_smem = 0;

// Asynchronous entry points run on the caller's stream; NULL is the CUDA
// default (legacy) stream.
cudaStream_t pick_stream(const ftlm_system*, void* st) { return reinterpret_cast<cudaStream_t>(st); }

int vchunk(int c64, int R) { return (c64 && R % 2 == 0) ? 2 : 1; }
int max_vectors(int c64) { return c64 ? 512 : 256; }

ftlm_status prepare_smem(size_t smem) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (smem <= g_prepared_smem) return FTLM_OK;
  CKI(prepare_rows_kernels(smem));
  g_prepared_smem = smem;
  return FTLM_OK;
}

// ---- launch shapes and the autotuner ----------------------------------------

struct ShapeKey {
  int n, qmax, R, c64;
  long long dim;
  bool operator<(const ShapeKey& o) const {
    return std::tie(n, qmax, R, c64, dim) < std::tie(o.n, o.qmax, o.R, o.c64, o.dim);
  }
};
std::map<ShapeKey, Shape> g_shapes;

// a launch shape set by ftlm_tune_shape or the autotuner for this system shape
bool has_shape_override(const ftlm_system* s, int R, int c64) {
  ShapeKey key{s->hs.n, s->hs.qmax, R, c64, (long long)s->hs.dim};
  std::lock_guard<std::mutex> lk(g_mu);
  return g_shapes.count(key) != 0;
}

Shape shape_for(int R, int c64, int threads_target, int tile_factor) {
  const int V = vchunk(c64, R);
  const int C = R / V;
  Shape sh;
  sh.threads = C * std::max(1, threads_target / C);
  const int rows_pass = sh.threads / C;
  int rows = std::max(rows_pass, (16384 / std::max(1, R)) * tile_factor);
  sh.rows_per_tile = ((rows + rows_pass - 1) / rows_pass) * rows_pass;
  sh.ctas_per_sm = 0;  // from the occupancy calculator
  return sh;
}

Shape default_shape(int R, int c64) { return shape_for(R, c64, 256, 1); }

InstDesc base_desc(const ftlm_system* s, int c64) {
  InstDesc d;
  const HostSystem& hs = s->hs;
  d.tab = c64 ? s->tab_f.p : s->tab_d.p;
  d.stride = reinterpret_cast<const long long*>(s->stride.p);
  d.q = reinterpret_cast<const int*>(s->q.p);
  d.dim = (long long)hs.dim;
  d.n = hs.n;
  d.all_half = hs.all_half ? 1 : 0;
  d.lay = hs.lay;
  return d;
}

struct HalfPlan {
  bool on = false;
  bool vm = false;  // vector-major kernel: R instances of one vector each (nvg = R, Rg = 1)
  bool hybrid = false;  // vector-major two-pass form
  int real_pm = 0;
  int min_blocks = 2;
  int passes = 1;  // > 1: one launch per pass, cubes covering all bits
  int K = 3, Rg = 1, threads = 256, rows_per_tile = 0, grid = 0, nvg = 0, tiles_per_vg = 0;
  size_t smem = 0;
  int stream_rows = 0, stream_tiles_per_vg = 0, stream_grid = 0;  // vector-major streaming launches
  long long dim = 0;
};

struct Plan {
  int c64 = 0, R = 0, V = 1, C = 1;
  Shape sh;
  int grid = 0;
  size_t smem = 0;
  LaunchArgs base;
  std::vector<int> tile_start;
  HalfPlan half;  // spin-1/2 kernel for the H.v modes, when applicable
  int wideV = 0;  // general kernel: H.v with 4 or 8 complex64 vectors per thread (0 = off)
  // vector-major general plan (any spins, several systems): every vector of a
  // run contiguous; the streaming modes see one instance per (system, vector),
  // H.v runs rows_vm_kernel over groups of gvm_V vectors of one system
  bool gen_vm = false;
  int gvm_V = 1, gvm_groups = 0, gvm_ntiles = 0, gvm_rows = 0, gvm_grid = 0;
  int gvm_cube = 0;  // > 0: cube_gather_kernel with the top site's 2s+1 rows per thread
  size_t gvm_smem = 0;
  std::vector<int> tile_start_g;  // prefix sum of H.v tiles over the groups
};

// the run keeps each Lanczos vector contiguous
bool plan_vmaj(const Plan& pl) { return pl.half.vm || pl.gen_vm; }

int largest_divisor_at_most(int R, int cap) {
  for (int g = std::min(R, cap); g >= 1; --g)
    if (R % g == 0) return g;
  return 1;
}

// Spin-1/2 register-cube launch: K cube bits, Rg vectors per group, tile of
// rows_factor cubes per slot.
bool make_half(const ftlm_system* s, int R, int c64, int K, int Rg, int rows_factor, bool multipass, HalfPlan& h,
               int min_blocks = 2) {
  const HostSystem& hs = s->hs;
  if (!hs.all_half || hs.n < K + 2 || K < 2 || K > 4 || Rg < 1 || Rg > R) return false;
  h = HalfPlan();
  h.K = K;
  h.Rg = Rg;
  h.passes = multipass ? (hs.n + K - 1) / K : 1;
  h.min_blocks = multipass ? 1 : (min_blocks > 2 ? 3 : 2);
  h.real_pm = hs.real_pm ? 1 : 0;
  const int slots = std::max(1, 256 / Rg);
  h.threads = slots * Rg;
  long long rows = (long long)slots * (1ll << K) * rows_factor;
  rows = std::min<long long>(rows, (long long)hs.dim);
  rows = std::max<long long>(rows, 1ll << K);
  h.rows_per_tile = (int)rows;
  h.nvg = (R + Rg - 1) / Rg;
  h.tiles_per_vg = (int)(((long long)hs.dim + rows - 1) / rows);  // the last tile may be ragged
  const long long ntiles = (long long)h.tiles_per_vg * h.nvg;
  if (ntiles > (1ll << 30)) return false;
  h.smem = half_smem_bytes(hs.n, K, h.rows_per_tile, h.threads);
  if (h.smem > 200 * 1024) return false;
  if (prepare_half_kernels(std::max<size_t>(h.smem, 48 * 1024)) != 0) return false;
  const int per_sm = half_max_ctas_per_sm(K, c64, h.threads, h.smem, h.min_blocks, h.passes > 1, R);
  h.grid = (int)std::max<long long>(1, std::min<long long>(ntiles, (long long)std::max(1, device_sm_count()) * per_sm));
  h.on = true;
  return true;
}

// Vector-major spin-1/2 launch: K cube bits above the 5 lane bits, tiles of
// 8 warps x rows_factor slabs of 2^(5+K) rows, R tiles ranges (one per vector).
bool make_vm(const ftlm_system* s, int R, int c64, int K, int rows_factor, int min_blocks, bool multipass,
             HalfPlan& h, bool hybrid = false) {
  const HostSystem& hs = s->hs;
  if (!hs.all_half || K < 3 || K > 4 || hs.n < kVmLaneBits + K || rows_factor < 1) return false;
  if (hybrid && hs.n < kVmLaneBits + 2 * K) return false;  // the two cubes must not overlap
  if (hs.dim >= (1ull << 31)) return false;  // 32-bit element indices
  h = HalfPlan();
  h.vm = true;
  h.K = K;
  h.Rg = 1;
  h.passes = hybrid ? 2 : (multipass ? (hs.n - kVmLaneBits + K - 1) / K : 1);  // cubes cover bits [5, n)
  h.hybrid = hybrid;
  // 1: one 512-thread CTA per SM; 2 or 3: 256-thread CTAs (3 only in one pass)
  h.min_blocks = min_blocks == 1 ? 1 : (h.passes > 1 ? 2 : (min_blocks > 2 ? 3 : 2));
  h.real_pm = hs.real_pm ? 1 : 0;
  h.threads = h.min_blocks == 1 ? 512 : 256;
  const long long slab = 1ll << (kVmLaneBits + K);
  long long rows = (long long)(h.threads / 32) * slab * rows_factor;
  rows = std::min<long long>(rows, (long long)hs.dim);  // dim and rows are powers of two >= slab
  h.rows_per_tile = (int)rows;
  h.nvg = R;
  h.dim = (long long)hs.dim;
  h.tiles_per_vg = (int)((long long)hs.dim / rows);  // per vector and pass
  const long long ntiles = (long long)h.tiles_per_vg * R * h.passes;
  if (ntiles > (1ll << 30)) return false;
  h.smem = vm_smem_bytes(hs.n, K, h.threads, h.passes, c64);
  if (h.smem > 200 * 1024) return false;
  if (prepare_vm_kernels(std::max<size_t>(h.smem, 48 * 1024)) != 0) return false;
  // the register budget allows min_blocks CTAs per SM: keep only their shared memory, the rest is L1
  if (set_vm_carveout(K, c64, h.passes > 1, h.min_blocks, h.smem, h.min_blocks) != 0) return false;
  const int per_sm = vm_max_ctas_per_sm(K, h.min_blocks, c64, h.threads, h.smem, h.passes > 1);
  const long long sms = std::max(1, device_sm_count());
  h.grid = (int)std::max<long long>(1, std::min<long long>(ntiles, sms * per_sm));
  h.stream_rows = (int)std::min<long long>(16384, (long long)hs.dim);
  h.stream_tiles_per_vg = (int)((long long)hs.dim / h.stream_rows);
  // two 256-thread CTAs per SM keep enough loads in flight for HBM and give
  // the last CTA half the partials of four (measured: 2.7 ms less per
  // 200-step run at d = 2^20, R = 64; one CTA per SM was 15 ms more)
  h.stream_grid = (int)std::max<long long>(1, std::min<long long>((long long)h.stream_tiles_per_vg * R, sms * 2));
  h.on = true;
  return true;
}

// General row-kernel launch over the instances `sys` (R vectors each).
ftlm_status make_general(const std::vector<ftlm_system*>& sys, int R, int c64, Plan& pl) {
  pl.V = vchunk(c64, R);
  pl.C = R / pl.V;
  LaunchArgs a;
  a.R = R;
  a.C = pl.C;
  a.rows_per_tile = pl.sh.rows_per_tile;
  int tab = 0, maxn = 0;
  pl.tile_start.assign(1, 0);
  for (auto* s : sys) {
    tab = std::max(tab, s->hs.lay.total);
    maxn = std::max(maxn, s->hs.n);
    const long long tiles = ((long long)s->hs.dim + a.rows_per_tile - 1) / a.rows_per_tile;
    if (pl.tile_start.back() + tiles > (1ll << 30)) return fail(FTLM_ERR_UNSUPPORTED, "too many tiles");
    pl.tile_start.push_back(pl.tile_start.back() + (int)tiles);
  }
  a.tab_reals = tab;
  a.max_n = maxn;
  a.n_inst = (int)sys.size();
  a.ntiles = pl.tile_start.back();
  pl.smem = rows_smem_bytes(a, c64, pl.sh.threads);
  if (pl.smem > 227 * 1024) return fail(FTLM_ERR_UNSUPPORTED, "coupling tables do not fit in shared memory");
  ftlm_status ps = prepare_smem(std::max<size_t>(pl.smem, 48 * 1024));
  if (ps != FTLM_OK) return ps;
  // H.v with more vectors per thread: the matrix elements of a row are computed
  // once for 4 or 8 vectors instead of 2 (complex64; the same tiles)
  pl.wideV = 0;
  if (c64 && R >= 4 && R % 4 == 0) {
    const int Vw = R % 8 == 0 ? 8 : 4, Cw = R / Vw;
    // (H.v keeps no reduction space in shared memory, so pl.smem covers it)
    if (pl.sh.threads % Cw == 0 && pl.sh.rows_per_tile % (pl.sh.threads / Cw) == 0) pl.wideV = Vw;
  }
  // the grid fills the SMs with the kernel that carries H.v.  The wide H.v
  // kernel runs two CTAs per SM while a system's block fits in the L2
  // (its gathers are served on chip and more L1 per tile pays), and as many as
  // fit once the block spills to HBM (the gathers' latency wants the warps).
  int per_sm = pl.sh.ctas_per_sm > 0 ? pl.sh.ctas_per_sm : rows_max_ctas_per_sm(c64, pl.sh.threads, pl.smem, pl.wideV);
  if (pl.sh.ctas_per_sm <= 0 && pl.wideV) {
    long long maxdim = 0;
    for (auto* s : sys) maxdim = std::max(maxdim, (long long)s->hs.dim);
    const long long block_bytes = maxdim * R * 8;
    if (block_bytes <= device_l2_bytes()) per_sm = std::min(per_sm, 2);
  }
  const int sms = std::max(1, device_sm_count());
  pl.grid = std::max(1, std::min(a.ntiles, sms * per_sm));
  pl.base = a;
  return FTLM_OK;
}

// allow_vm: the caller keeps its Lanczos block vector-major (ftlm_run); for
// row-major blocks a vector-major shape falls back to the row-major cube kernel.
ftlm_status make_plan(const std::vector<ftlm_system*>& sys, int R, int c64, Plan& pl, const Shape* force = nullptr,
                      bool allow_vm = false) {
  pl.c64 = c64;
  pl.R = R;
  const ftlm_system* big = sys[0];
  for (auto* s : sys)
    if (s->hs.dim > big->hs.dim) big = s;
  if (force) {
    pl.sh = *force;
  } else {
    ShapeKey key{big->hs.n, big->hs.qmax, R, c64, (long long)big->hs.dim};
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_shapes.find(key);
    pl.sh = it != g_shapes.end() ? it->second : default_shape(R, c64);
  }
  pl.half.on = false;
  if (sys.size() == 1 && pl.sh.half_K > 0 && pl.sh.half_vm && allow_vm &&
      make_vm(sys[0], R, c64, pl.sh.half_K, pl.sh.half_rows, pl.sh.half_min_blocks, pl.sh.half_multipass != 0,
              pl.half, pl.sh.half_hybrid != 0)) {
    // the streaming modes see R one-vector instances of the same system
    const Shape keep = pl.sh;
    pl.sh = default_shape(1, c64);
    ftlm_status gs = make_general(std::vector<ftlm_system*>(R, sys[0]), 1, c64, pl);
    pl.sh.half_K = keep.half_K;
    pl.sh.half_vm = 1;
    return gs;
  }
  if (sys.size() == 1 && allow_vm && !force && pl.sh.half_K == 0 && !pl.sh.explicit_general) {
    // default for runs on spin-1/2 systems: the vector-major single-pass gather
    const int K = c64 ? 4 : 3;  // complex128 cubes of 16 rows spill at 128 registers
    // one 512-thread CTA per SM (one copy of the tables, more L1), tiles of 2 units per warp
    if (make_vm(sys[0], R, c64, K, 2, 1, false, pl.half)) {
      pl.sh = default_shape(1, c64);
      ftlm_status gs = make_general(std::vector<ftlm_system*>(R, sys[0]), 1, c64, pl);
      pl.sh.half_K = K;
      pl.sh.half_vm = 1;
      return gs;
    }
  }
  // runs on other systems and batches: the vector-major general gather by
  // default when it can hold the top site's rows as a register cube (every
  // system with the same top spin, a group size dividing R), or when the
  // largest system's block of R vectors fits in L2; else the row-major one.
  // Measured on GB300: with one row a thread the vector-major gather is 24 %
  // faster than the row-major one on s = 1 chains whose largest block is
  // 68 MB but 5 % slower on a 150 MB mixed-spin block, where the cube form is
  // 17 % faster than both.  An autotuned or forced shape decides for itself.
  int Qtop = sys[0]->hs.n >= 2 ? sys[0]->hs.q.back() : 0;
  for (auto* s : sys)
    if (s->hs.n < 2 || s->hs.q.back() != Qtop) Qtop = 0;
  // the cube's group size: the default for the top spin, else 4, whichever
  // has a kernel and divides R (0: none)
  auto cube_group = [&](int want) {
    if (!Qtop) return 0;
    if (want > 0) return (cube_vectors(Qtop, c64, want) && R % want == 0) ? want : 0;
    for (int v : {cube_vectors(Qtop, c64), 4})
      if (v > 0 && cube_vectors(Qtop, c64, v) && R % v == 0) return v;
    return 0;
  };
  const int Vdef = cube_group(0);
  const bool gvm_fits = (long long)big->hs.dim * R * (c64 ? 8 : 16) <= device_l2_bytes();
  const bool gvm_default = gvm_fits || Vdef > 0;
  const bool want_gvm = pl.sh.general_vm == 1 || (pl.sh.general_vm < 0 && !force && gvm_default);
  if (allow_vm && want_gvm && pl.sh.half_K == 0 && !pl.sh.explicit_general) {
    int V = 1;
    for (int v : {8, 4, 2, 1})
      if (R % v == 0 && rows_vm_supported(v, c64)) {
        V = v;
        break;
      }
    // the register cube along the top site when every system has the same top
    // spin and a kernel exists for it and for a group size dividing R
    const int Q = Qtop;
    const int Vc = (Q && pl.sh.gvm_cube != 0) ? cube_group(std::max(0, pl.sh.gvm_cube)) : 0;
    const bool cube = Vc > 0;
    if (cube) V = Vc;
    std::vector<ftlm_system*> vecs;  // one instance per (system, vector), system-major
    for (auto* s : sys)
      for (int k = 0; k < R; ++k) vecs.push_back(s);
    const Shape keep = pl.sh;
    pl.sh = default_shape(1, c64);
    ftlm_status gs = make_general(vecs, 1, c64, pl);
    if (gs != FTLM_OK) return gs;
    pl.sh.half_K = keep.half_K;
    pl.gen_vm = true;
    pl.gvm_V = V;
    pl.gvm_cube = cube ? Q : 0;
    // 1024 rows: four a thread of a 256-thread CTA; with the cube, 256 bases
    // (one a thread: the CTAs then share the neighbourhoods they gather in L2)
    pl.gvm_rows = keep.gvm_rows > 0 && keep.general_vm == 1 ? keep.gvm_rows : (cube ? 256 : 1024);
    pl.tile_start_g.assign(1, 0);
    for (auto* s : sys)
      for (int g = 0; g < R / V; ++g) {
        const long long rows = cube ? (long long)s->hs.dim / Q : (long long)s->hs.dim;  // bases, or rows
        const long long tiles = (rows + pl.gvm_rows - 1) / pl.gvm_rows;
        if (pl.tile_start_g.back() + tiles > (1ll << 30)) return fail(FTLM_ERR_UNSUPPORTED, "too many tiles");
        pl.tile_start_g.push_back(pl.tile_start_g.back() + (int)tiles);
      }
    pl.gvm_groups = (int)pl.tile_start_g.size() - 1;
    pl.gvm_ntiles = pl.tile_start_g.back();
    int per_sm = 1;
    if (cube) {
      pl.gvm_smem = gather_smem_bytes(pl.base, c64, 256);  // tables and per-thread columns, no reduction space
      CKI(prepare_cube(Q, V, c64, std::max<size_t>(pl.gvm_smem, 48 * 1024)));
      per_sm = cube_ctas_per_sm(Q, V, c64, 256, pl.gvm_smem);
    } else {
      pl.gvm_smem = pl.smem;  // the same tables and per-thread columns as the streaming plan
      CKI(prepare_rows_vm(V, c64, std::max<size_t>(pl.gvm_smem, 48 * 1024)));
      per_sm = rows_vm_ctas_per_sm(V, c64, 256, pl.gvm_smem);
    }
    pl.gvm_grid = std::max(1, std::min(pl.gvm_ntiles, std::max(1, device_sm_count()) * per_sm));
    return FTLM_OK;
  }
  ftlm_status gs = make_general(sys, R, c64, pl);
  if (gs != FTLM_OK) return gs;
  if (sys.size() == 1 && pl.sh.half_K > 0 && !pl.sh.half_vm)
    make_half(sys[0], R, c64, pl.sh.half_K, pl.sh.Rg, pl.sh.half_rows, pl.sh.half_multipass != 0, pl.half,
              pl.sh.half_min_blocks);
  else if (sys.size() == 1 && (!force || pl.sh.half_vm) && !pl.sh.explicit_general && sys[0]->hs.all_half)
    make_half(sys[0], R, c64, 3, largest_divisor_at_most(R, 16), 4, false, pl.half);
  return FTLM_OK;
}

// Launches one mode of the plan: the spin-1/2 kernel for H.v modes when the
// plan has it, the general row kernel otherwise.
int launch_plan(const Plan& pl, LaunchArgs a, void* st) {
  if (pl.gen_vm && a.mode == kModeApply) {  // the groups' tile list follows the instances' in the same buffer
    a.n_inst = pl.gvm_groups;
    a.ntiles = pl.gvm_ntiles;
    a.rows_per_tile = pl.gvm_rows;
    if (!a.inline_one) a.tile_start += pl.base.n_inst + 1;
    if (pl.gvm_cube) return launch_cube(a, pl.gvm_cube, pl.gvm_V, pl.c64, pl.gvm_grid, 256, pl.gvm_smem, st);
    return launch_rows_vm(a, pl.gvm_V, pl.c64, pl.gvm_grid, 256, pl.gvm_smem, st);
  }
  if (pl.half.on && pl.half.vm &&
      (a.mode == kModeStep || a.mode == kModeStartNorm || a.mode == kModeUpdate || a.mode == kModeApplyS)) {
    a.rows_per_tile = pl.half.stream_rows;
    a.tiles_per_vg = pl.half.stream_tiles_per_vg;
    a.n_inst = pl.half.nvg;
    a.ntiles = pl.half.stream_tiles_per_vg * pl.half.nvg;
    a.inline_one = 0;
    return launch_vm_stream(a, pl.c64, pl.half.stream_grid, st);
  }
  if (pl.half.on && pl.half.vm && a.mode == kModeApply) {  // a.inst: R one-vector instances
    a.rows_per_tile = pl.half.rows_per_tile;
    a.tiles_per_vg = pl.half.tiles_per_vg;
    a.nvg = pl.half.nvg;
    a.n_inst = pl.half.nvg;
    a.ntiles = pl.half.tiles_per_vg * pl.half.nvg;
    a.real_pm = pl.half.real_pm;
    a.min_blocks = pl.half.min_blocks;
    // one vector, or a regular block (vm_stride): the descriptor by value
    a.inline_one = (a.inline_one && (pl.half.nvg == 1 || a.vm_stride)) ? 1 : 0;
    a.pass_stride = (long long)pl.half.nvg * pl.half.dim;
    if (pl.half.hybrid) {  // two launches: the bottom cube (one-pass kernel), then the top cube adds its terms
      LaunchArgs b = a;
      b.single_pass = 1;
      b.hybrid = 1;
      b.npass = 1;
      b.gather_alpha = 0;
      b.ntiles = pl.half.tiles_per_vg * pl.half.nvg;
      const int e = launch_vm(b, pl.half.K, pl.half.min_blocks, pl.c64, pl.half.grid, pl.half.threads, pl.half.smem, st);
      if (e) return e;
      a.single_pass = 0;
      a.hybrid = 2;
      a.npass = 1;
      a.ntiles = pl.half.tiles_per_vg * pl.half.nvg;
      return launch_vm(a, pl.half.K, pl.half.min_blocks, pl.c64, pl.half.grid, pl.half.threads, pl.half.smem, st);
    }
    a.single_pass = pl.half.passes == 1 ? 1 : 0;
    a.npass = pl.half.passes;  // pass p writes y + p * R * d (vector-major blocks)
    a.hybrid = 0;
    a.ntiles = pl.half.tiles_per_vg * pl.half.nvg * pl.half.passes;
    return launch_vm(a, pl.half.K, pl.half.min_blocks, pl.c64, pl.half.grid, pl.half.threads, pl.half.smem, st);
  }
  const bool half = pl.half.on && !pl.half.vm &&
                    (a.mode == kModeApply || (a.mode == kModeLanczos && pl.half.passes == 1));
  if (half) {
    a.rows_per_tile = pl.half.rows_per_tile;
    a.Rg = pl.half.Rg;
    a.nvg = pl.half.nvg;
    a.tiles_per_vg = pl.half.tiles_per_vg;
    a.ntiles = pl.half.tiles_per_vg * pl.half.nvg;
    a.real_pm = pl.half.real_pm;
    a.min_blocks = pl.half.min_blocks;
    const int K = pl.half.K;
    const int n = pl.base.max_n;
    if (pl.half.passes == 1) {
      a.single_pass = 1;
      return launch_half(a, K, pl.c64, pl.half.grid, pl.half.threads, pl.half.smem, st);
    }
    for (int p = 0; p < pl.half.passes; ++p) {  // cubes [min(pK, n-K), +K) cover every bit
      a.cube_lo = std::min(p * K, n - K);
      a.new_lo = p * K;
      a.later_lo = a.cube_lo + K;
      a.first_pass = p == 0;
      a.single_pass = 0;
      const int e = launch_half(a, K, pl.c64, pl.half.grid, pl.half.threads, pl.half.smem, st);
      if (e) return e;
    }
    return 0;
  }
  if (pl.wideV && a.mode == kModeApply) {
    a.C = a.R / pl.wideV;
    return launch_rows_wide(a, pl.wideV, pl.grid, pl.sh.threads, pl.smem, st);
  }
  // the streaming modes need far fewer CTAs than the gathers to saturate HBM,
  // and fewer CTAs means fewer partial sums for the last CTA to add up
  const bool streaming = a.mode == kModeEpilogue || a.mode == kModeUpdate || a.mode == kModeStartNorm ||
                         a.mode == kModeScale || a.mode == kModeStep;
  const int grid = streaming ? std::min(pl.grid, 2 * std::max(1, device_sm_count())) : pl.grid;
  return launch_rows(a, pl.c64, grid, pl.sh.threads, pl.smem, st);
}

// The Lanczos step of the plan runs as the vector-major one-pass gather with
// the step's w' in its epilogue, then the update pass (see enqueue_run).
bool vm_fused_step(const Plan& pl) { return pl.half.on && pl.half.vm && pl.half.passes == 1 && !pl.half.hybrid; }

// The per-unit coefficient tables of the one-pass vector-major gather with K
// cube bits, built once per system (and rebuilt for another K or precision)
// on stream st; their pointer is baked into captured graphs, so a rebuild
// bumps the system's generation.
ftlm_status ensure_unit_tables(ftlm_system* s, int K, int c64, cudaStream_t st) {
  DevBuf& b = s->ut[c64 ? 1 : 0];
  if (b.p && s->ut_K[c64 ? 1 : 0] == K) return FTLM_OK;
  const int n = s->hs.n;
  const long long nunits = (long long)(s->hs.dim >> (kVmLaneBits + K));
  const size_t bytes = (size_t)nunits * vm_unit_table_stride(n, K) * (c64 ? 4 : 8);
  if (b.p) CK(cudaDeviceSynchronize());  // a rebuild: no launch may still read the old tables
  b.release();
  CK(b.ensure(bytes));
  CKI(launch_vm_unit_tables(reinterpret_cast<const double*>(s->tab_d.p), s->hs.lay, n, K, nunits, b.p, c64, st));
  s->ut_K[c64 ? 1 : 0] = K;
  s->gen++;
  return FTLM_OK;
}

int plan_max_grid(const Plan& pl) {
  return std::max(std::max(pl.grid, pl.gen_vm ? pl.gvm_grid : 0),
                  pl.half.on ? std::max(pl.half.grid, pl.half.stream_grid) : 0);
}

// ---- workspace ----------------------------------------------------------------

size_t scalar_bytes(int R, int M) {
  return sizeof(double) * ((size_t)M * R * 4 + (size_t)(M + 1) * R + R) + sizeof(int) * 2 * (size_t)R + 64;
}

ftlm_status ensure_workspace(ftlm_system* s, int R, int M, int c64) {
  const size_t block = (size_t)s->hs.dim * R * (c64 ? 8 : 16);
  if (s->A.bytes < block || s->scal.bytes < scalar_bytes(R, M)) {
    s->A.release();
    s->B.release();
    s->U.release();
    s->scal.release();
    CK(s->A.ensure(block));
    CK(s->B.ensure(block));
    CK(s->U.ensure(block));
    CK(s->scal.ensure(scalar_bytes(R, M)));
    s->gen++;
  }
  return FTLM_OK;
}

// parts: H q_j blocks (one per pass of the vector-major multi-pass gather)
ftlm_status ensure_hq(ftlm_system* s, int R, int c64, int parts = 1) {
  const size_t block = (size_t)s->hs.dim * R * (c64 ? 8 : 16) * parts;
  if (s->Hq.bytes < block) {
    s->Hq.release();
    CK(s->Hq.ensure(block));
    s->gen++;
  }
  return FTLM_OK;
}

DevScalars scalars_at(void* base, int R, int M) {
  DevScalars sc;
  sc.ss = R;
  double* b = reinterpret_cast<double*>(base);
  sc.alpha = b;
  b += (size_t)M * R;
  sc.beta = b;
  b += (size_t)M * R;
  sc.p = b;
  b += (size_t)M * R * 2;
  sc.sigma = b;
  b += (size_t)(M + 1) * R;
  sc.scale = b;
  b += R;
  int* ib = reinterpret_cast<int*>(b);
  sc.active = ib;
  sc.meff = ib + R;
  return sc;
}

// The scalars of vector k alone, as a one-vector instance sees them (row
// stride R in the shared arrays).
DevScalars scalars_of_vector(void* base, int R, int M, int k) {
  DevScalars sc = scalars_at(base, R, M);
  sc.alpha += k;
  sc.beta += k;
  sc.p += 2 * k;
  sc.sigma += k;
  sc.scale += k;
  sc.active += k;
  sc.meff += k;
  return sc;
}

// ---- captured runs ------------------------------------------------------------

struct RunCtx {
  std::string key;
  std::vector<uint64_t> deps;  // system ids
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  DevBuf desc, tiles, partials, counter;
  std::vector<cudaEvent_t> ev;  // [2M + 2] when kernel timing is on
  int launches = 0, hv_launches = 0;
  char* pinned = nullptr;
  size_t h2d = 0;
  ~RunCtx() {
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    desc.release();
    tiles.release();
    partials.release();
    counter.release();
    for (auto e : ev) cudaEventDestroy(e);
    if (pinned) cudaFreeHost(pinned);
  }
};

std::vector<std::unique_ptr<RunCtx>> g_ctx;  // small cache of captured runs, newest last

void purge_ctx_of(uint64_t id) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_ctx.begin(); it != g_ctx.end();) {
    bool hit = false;
    for (auto d : (*it)->deps) hit = hit || d == id;
    if (hit) it = g_ctx.erase(it);
    else ++it;
  }
}

std::string run_key(const std::vector<ftlm_system*>& sys, const ftlm_run_params* p, const Plan& pl) {
  char buf[640];
  std::string k;
  for (auto* s : sys) {
    snprintf(buf, sizeof buf, "%llu:%llu,", (unsigned long long)s->id, (unsigned long long)s->gen);
    k += buf;
  }
  double u[3];
  observable_coefs(sys[0]->hs, p->obs_dir, u);
  snprintf(buf, sizeof buf,
           "|R%d M%d dt%d seed%llu off%llu st%d bo%llu us%p tk%d th%d rpt%d g%d tol%.17g obs%.17g,%.17g,%.17g,%d s%p",
           p->R, p->M, (int)p->dtype, (unsigned long long)p->seed, (unsigned long long)p->vec_offset, p->start,
           (unsigned long long)p->basis_offset, p->user_start, p->time_kernels, pl.sh.threads, pl.sh.rows_per_tile,
           pl.grid, p->breakdown_tol, u[0], u[1], u[2], p->obs_dir ? 1 : 0, p->stream);
  k += buf;
  k += p->symmetric ? "|sym" : "";
  k += p->reorth ? "|reorth" : "";
  k += pl.gen_vm ? "|gvm" + std::to_string(pl.gvm_V) + "x" + std::to_string(pl.gvm_rows) + "c" +
                       std::to_string(pl.gvm_cube)
                 : "";
  snprintf(buf, sizeof buf, "|half%d vm%d hy%d K%d Rg%d rpt%d g%d P%d mb%d", pl.half.on ? 1 : 0, pl.half.vm ? 1 : 0,
           pl.half.hybrid ? 1 : 0,
           pl.half.K, pl.half.Rg, pl.half.rows_per_tile, pl.half.grid, pl.half.passes, pl.half.min_blocks);
  return k + buf;
}

ftlm_status validate_params(const ftlm_run_params* p, const std::vector<ftlm_system*>& sys) {
  if (!p) return fail(FTLM_ERR_INVALID_ARG, "params is NULL");
  if (p->dtype != FTLM_C64 && p->dtype != FTLM_C128) return fail(FTLM_ERR_INVALID_ARG, "unknown dtype");
  const int c64 = p->dtype == FTLM_C64;
  if (p->R < 1 || p->R > max_vectors(c64))
    return fail(FTLM_ERR_INVALID_ARG, "R must be in 1.." + std::to_string(max_vectors(c64)));
  if (p->M < 1 || p->M > 100000) return fail(FTLM_ERR_INVALID_ARG, "M must be in 1..100000");
  if (!p->T || p->nT < 1) return fail(FTLM_ERR_INVALID_ARG, "temperature grid missing");
  for (int t = 0; t < p->nT; ++t)
    if (!(p->T[t] > 0.0) || !std::isfinite(p->T[t])) return fail(FTLM_ERR_INVALID_ARG, "temperatures must be > 0");
  if (p->start < 0 || p->start > 3) return fail(FTLM_ERR_INVALID_ARG, "unknown start mode");
  if (p->start == FTLM_START_USER && !p->user_start) return fail(FTLM_ERR_INVALID_ARG, "user_start is NULL");
  if (p->start == FTLM_START_USER && (reinterpret_cast<uintptr_t>(p->user_start) & 15))
    return fail(FTLM_ERR_INVALID_ARG, "user_start must be 16-byte aligned");
  if (p->start == FTLM_START_USER && sys.size() != 1)
    return fail(FTLM_ERR_INVALID_ARG, "user start vectors need a single system");
  if (p->symmetric && sys.size() != 1) return fail(FTLM_ERR_INVALID_ARG, "symmetric runs take one system");
  if (p->symmetric != 0 && p->symmetric != 1) return fail(FTLM_ERR_INVALID_ARG, "symmetric must be 0 or 1");
  if (p->reorth != 0 && p->reorth != 1) return fail(FTLM_ERR_INVALID_ARG, "reorth must be 0 or 1");
  if (p->reorth && sys.size() != 1)
    return fail(FTLM_ERR_UNSUPPORTED, "re-orthogonalised runs take one system (ftlm_run)");
  if (!(p->breakdown_tol >= 0) || !std::isfinite(p->breakdown_tol))
    return fail(FTLM_ERR_INVALID_ARG, "breakdown_tol must be finite and >= 0");
  if (p->obs_dir && !(std::isfinite(p->obs_dir[0]) && std::isfinite(p->obs_dir[1]) && std::isfinite(p->obs_dir[2])))
    return fail(FTLM_ERR_INVALID_ARG, "obs_dir must be finite");
  for (auto* s : sys) {
    if (!s) return fail(FTLM_ERR_INVALID_ARG, "system is NULL");
    if (p->start == FTLM_START_BASIS && p->basis_offset + (uint64_t)p->R > s->hs.dim)
      return fail(FTLM_ERR_INVALID_ARG, "basis_offset + R exceeds the dimension");
  }
  return FTLM_OK;
}

// Staged per system: alpha, beta, p ([M][R], [M][R], [M][R][2]) and sigma ([M][R],
// the scale of the unnormalised Lanczos vectors), contiguous in the scalars;
// then M_eff [R].
size_t staged_doubles(int R, int M) { return (size_t)M * R * 5; }
size_t staged_bytes(int R, int M) { return sizeof(double) * staged_doubles(R, M) + sizeof(int) * (size_t)R; }

// Enqueues one whole run on `st` (which the caller is capturing).
ftlm_status enqueue_run(RunCtx& ctx, const std::vector<ftlm_system*>& sys, const ftlm_run_params* p, const Plan& pl,
                        cudaStream_t st) {
  const int M = p->M, R = p->R, c64 = pl.c64;
  const int n = (int)sys.size();
  const int nd = plan_vmaj(pl) ? n * R : n;  // descriptors per kind: one per (system, vector) in the vector-major layout
  const InstDesc* d_even = reinterpret_cast<const InstDesc*>(ctx.desc.p);
  const InstDesc* d_odd = d_even + nd;
  const InstDesc* d_start = d_even + 2 * nd;
  const InstDesc* d_gather_even = d_even + 3 * nd;  // split steps: x = q_j, y = Hq
  const InstDesc* d_gather_odd = d_even + 4 * nd;
  // the spin-1/2 gathers and the wide general gather run alone; the step epilogue streams afterwards
  const bool split = pl.half.on || pl.wideV || pl.gen_vm;
  // single-pass gathers also sum Re<q_j|H q_j>, so alpha_j is known before the
  // epilogue, which then finishes the step in one pass (no separate update)
  const bool fused = pl.half.on && (pl.half.passes == 1 || pl.half.vm);
  // the vector-major one-pass gather goes further: it writes w' over q_{j-1}
  // and sums alpha_j and p_j itself; the update pass finishes the step
  const bool fused_step = vm_fused_step(pl);
  LaunchArgs a = pl.base;
  a.tile_start = reinterpret_cast<const int*>(ctx.tiles.p);
  a.partials = reinterpret_cast<double*>(ctx.partials.p);
  a.counter = reinterpret_cast<unsigned*>(ctx.counter.p);
  if (fused_step) a.unit_tab = sys[0]->ut[c64 ? 1 : 0].p;  // built by run_impl before the capture
  ctx.launches = 0;
  ctx.hv_launches = 0;
  const bool tk = p->time_kernels != 0;
  int evi = 0;
  if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
  const int vmaj = plan_vmaj(pl) ? 1 : 0;
  for (int k = 0; k < n; ++k) {  // start block -> A
    InstDesc h = base_desc(sys[k], c64);
    const long long dim = (long long)sys[k]->hs.dim;
    if (p->start == FTLM_START_RANDOM)
      CKI(launch_start_random(&h, nullptr, R, p->seed, p->vec_offset, sys[k]->A.p, c64, st, vmaj));
    else if (p->start == FTLM_START_PAIRS)
      CKI(launch_start_pairs(&h, R, p->seed, p->vec_offset, sys[k]->A.p, c64, st, vmaj));
    else if (p->start == FTLM_START_BASIS)
      CKI(launch_start_basis(dim, R, p->basis_offset, sys[k]->A.p, c64, st, vmaj));
    else if (vmaj)
      CKI(launch_to_vector_major(p->user_start, sys[k]->A.p, dim, R, c64, st));
    else
      CKI(launch_copy_block(p->user_start, sys[k]->A.p, (size_t)dim * R * (c64 ? 8 : 16), st));
    ctx.launches++;
  }
  a.inst = d_start;  // sigma_0 = 1/|q_0|, then U = sigma_0 (u.S) q_0
  a.mode = kModeStartNorm;
  CKI(launch_plan(pl, a, st));
  a.mode = kModeApplyS;
  a.use_sigma0 = 1;
  CKI(launch_plan(pl, a, st));
  a.use_sigma0 = 0;
  ctx.launches += 2;
  for (int j = 0; j < M; ++j) {
    a.inst = (j % 2 == 0) ? d_even : d_odd;
    a.step = j;
    a.first = j == 0;
    // time_kernels: events at the step's start and end and around its H.v launch
    // ([1 + 4j] .. [4 + 4j]); a step's start event follows the previous step's
    // end event with no work between them, so their difference is the gap
    // between two launches of the graph
    if (tk) {
      evi = 1 + 4 * j;
      CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
    }
    if (p->symmetric || p->reorth) {  // keep q_j (vector-major): the matrix of u.S in the Lanczos basis, or
                                       // the vectors the next ones are re-orthogonalised against
      ftlm_system* s0 = sys[0];
      const size_t vb = (size_t)s0->hs.dim * R * (c64 ? 8 : 16);
      const void* q = (j % 2 == 0) ? s0->A.p : s0->B.p;
      void* dst = static_cast<char*>(s0->Vs.p) + vb * j;
      if (plan_vmaj(pl)) CK(cudaMemcpyAsync(dst, q, vb, cudaMemcpyDeviceToDevice, st));
      else CKI(launch_to_vector_major(q, dst, (long long)s0->hs.dim, R, c64, st));
      ctx.launches++;
    }
    if (fused_step) {
      LaunchArgs g = a;  // x = q_j, y = q_{j-1} (w' in place), u
      g.mode = kModeApply;
      g.fused_step = 1;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      CKI(launch_plan(pl, g, st));
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      a.mode = kModeUpdate;
      CKI(launch_plan(pl, a, st));
      ctx.launches += 2;
      ctx.hv_launches++;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[4 + 4 * j], st, cudaEventRecordExternal));
      continue;
    }
    if (pl.gen_vm && pl.gvm_cube) {  // the cube gather writes w' over q_{j-1} and sets alpha_j, p_j
      LaunchArgs g = a;  // x = q_j, y = q_{j-1}, u
      g.mode = kModeApply;
      g.fused_step = 1;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      CKI(launch_plan(pl, g, st));
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      a.mode = kModeUpdate;
      CKI(launch_plan(pl, a, st));
      ctx.launches += 2;
      ctx.hv_launches++;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[4 + 4 * j], st, cudaEventRecordExternal));
      continue;
    }
    if (split) {
      LaunchArgs g = a;
      g.inst = (j % 2 == 0) ? d_gather_even : d_gather_odd;
      g.mode = kModeApply;
      g.gather_alpha = fused ? 1 : 0;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      CKI(launch_plan(pl, g, st));
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      if (fused) {
        a.mode = kModeStep;
        a.hq_parts = (pl.half.vm && !pl.half.hybrid) ? pl.half.passes : 1;  // the passes' partial H q_j blocks
        a.hq_stride = (long long)R * (long long)sys[0]->hs.dim;
        CKI(launch_plan(pl, a, st));
        a.hq_parts = 1;
        ctx.launches += 2;
        ctx.hv_launches++;
        if (tk) CK(cudaEventRecordWithFlags(ctx.ev[4 + 4 * j], st, cudaEventRecordExternal));
        continue;
      }
      a.mode = kModeEpilogue;
      CKI(launch_plan(pl, a, st));
      ctx.launches++;
    } else {
      a.mode = kModeLanczos;
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
      CKI(launch_plan(pl, a, st));
      if (tk) CK(cudaEventRecordWithFlags(ctx.ev[evi++], st, cudaEventRecordExternal));
    }
    a.mode = kModeUpdate;
    CKI(launch_plan(pl, a, st));
    ctx.launches += 2;
    ctx.hv_launches++;
    if (p->reorth) {  // two Gram-Schmidt passes against q_0..q_j, then the norm of what is left
      ftlm_system* s0 = sys[0];
      const DevScalars sc = scalars_at(s0->scal.p, R, M);
      void* w = (j % 2 == 0) ? s0->B.p : s0->A.p;
      for (int pass = 0; pass < 2; ++pass)
        CKI(launch_reorth_pass(s0->Vs.p, w, (long long)s0->hs.dim, R, j, M, reinterpret_cast<double*>(s0->Gre.p),
                               sc.sigma, c64, st));
      a.mode = kModeUpdate;
      a.update_no_alpha = 1;
      CKI(launch_plan(pl, a, st));
      a.update_no_alpha = 0;
      ctx.launches += 5;
    }
    if (tk) CK(cudaEventRecordWithFlags(ctx.ev[4 + 4 * j], st, cudaEventRecordExternal));
  }
  if (tk) CK(cudaEventRecordWithFlags(ctx.ev[4 * M + 1], st, cudaEventRecordExternal));
  const size_t per = staged_bytes(R, M);
  for (int k = 0; k < n; ++k) {  // alpha, beta, p, M_eff -> pinned host staging
    DevScalars sc = scalars_at(sys[k]->scal.p, R, M);
    char* dst = ctx.pinned + per * k;
    CK(cudaMemcpyAsync(dst, sc.alpha, sizeof(double) * staged_doubles(R, M), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(dst + sizeof(double) * staged_doubles(R, M), sc.meff, sizeof(int) * R, cudaMemcpyDeviceToHost,
                       st));
  }
  return FTLM_OK;
}

ftlm_status build_ctx(RunCtx& c, const std::vector<ftlm_system*>& sys, const ftlm_run_params* p, const Plan& pl,
                      cudaStream_t st) {
  const int c64 = pl.c64, R = p->R, M = p->M, n = (int)sys.size();
  for (auto* s : sys) c.deps.push_back(s->id);
  // descriptors: even steps (x = A, y = B), odd steps (x = B, y = A), start (x = A, y = U),
  // and for split steps the gathers (x = A or B, y = Hq); one per system, or in the
  // vector-major layout one per vector (pointers at vector k, scalars of vector k)
  const bool vmaj = plan_vmaj(pl);
  const int nd = vmaj ? n * R : n;
  std::vector<InstDesc> h(5 * nd);
  for (int k = 0; k < nd; ++k) {
    ftlm_system* s = sys[vmaj ? k / R : k];  // vector-major: instance k is vector k % R of system k / R
    const int vec = vmaj ? k % R : 0;
    InstDesc d = base_desc(s, c64);
    d.sc = vmaj ? scalars_of_vector(s->scal.p, R, M, vec) : scalars_at(s->scal.p, R, M);
    const size_t off = vmaj ? (size_t)vec * s->hs.dim * (c64 ? 8 : 16) : 0;  // bytes to vector vec
    char* A = static_cast<char*>(s->A.p) + off;
    char* B = static_cast<char*>(s->B.p) + off;
    char* U = static_cast<char*>(s->U.p) + off;
    char* Hq = s->Hq.p ? static_cast<char*>(s->Hq.p) + off : nullptr;
    d.u = U;
    d.M = M;
    d.tol = p->breakdown_tol > 0 ? p->breakdown_tol : (c64 ? 1e-6 : 1e-12);
    observable_coefs(s->hs, p->obs_dir, d.obs);  // per instance: each system has its own field direction
    InstDesc e = d, o = d, t = d;
    e.x = A;
    e.y = B;
    o.x = B;
    o.y = A;
    t.x = A;
    t.y = U;
    e.hq = o.hq = Hq;
    InstDesc ge = d, go = d;
    ge.x = A;
    ge.y = Hq;
    go.x = B;
    go.y = Hq;
    h[k] = e;
    h[nd + k] = o;
    h[2 * nd + k] = t;
    h[3 * nd + k] = ge;
    h[4 * nd + k] = go;
  }
  CK(c.desc.ensure(sizeof(InstDesc) * h.size()));
  CK(cudaMemcpy(c.desc.p, h.data(), sizeof(InstDesc) * h.size(), cudaMemcpyHostToDevice));
  std::vector<int> tiles = pl.tile_start;  // the instances' tile list, then the H.v groups' (vector-major general)
  tiles.insert(tiles.end(), pl.tile_start_g.begin(), pl.tile_start_g.end());
  CK(c.tiles.ensure(sizeof(int) * tiles.size()));
  CK(cudaMemcpy(c.tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice));
  CK(c.partials.ensure(sizeof(double) * (size_t)n * plan_max_grid(pl) * R * kNumPartials));  // n_inst x R = R x 1 when vector-major
  CK(c.counter.ensure(64));
  CK(cudaMemset(c.counter.p, 0, 64));
  c.h2d = sizeof(InstDesc) * h.size() + sizeof(int) * tiles.size();
  CK(cudaMallocHost(reinterpret_cast<void**>(&c.pinned), staged_bytes(R, M) * n));
  if (p->time_kernels) {
    c.ev.resize(4 * M + 2);
    for (auto& e : c.ev) CK(cudaEventCreate(&e));
  }
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  ftlm_status es = enqueue_run(c, sys, p, pl, st);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (es != FTLM_OK) {
    if (g) cudaGraphDestroy(g);
    return es;
  }
  CK(ce);
  c.g = g;
  CK(cudaGraphInstantiate(&c.ex, g, 0));
  return FTLM_OK;
}

// ---- symmetric estimator: O_ij = <v_i|u.S|v_j> per vector ---------------------

// After a symmetric run: G_r[i][j] = <q_i|u.S q_j> for the stored unnormalised
// vectors q_0 .. q_{M-1} of every vector r, in one fused kernel (u.S q_j is
// formed tile by tile in shared memory, never stored) plus a fixed-order
// reduction of its per-range partials; then O_ij = sigma_i sigma_j G_ij on
// the host.  Omat [R][M][M] complex row-major; sigma [M][R].
ftlm_status symmetric_matrices(ftlm_system* s, const ftlm_run_params* p, cudaStream_t st, const double* sigma,
                               std::vector<double>& Omat, double& ms) {
  const int R = p->R, M = p->M, c64 = p->dtype == FTLM_C64;
  const long long d = (long long)s->hs.dim;
  const int nranges = sym_ranges(d, R, M);
  const size_t pbytes = sizeof(double) * sym_partial_doubles(R, M, nranges);
  if (s->Wc.bytes < pbytes) {
    s->Wc.release();
    if (s->Wc.ensure(pbytes) != cudaSuccess) return fail(FTLM_ERR_OUT_OF_MEMORY, "O matrix partial sums");
  }
  const size_t obytes = sizeof(double) * 2 * (size_t)R * M * M;
  if (s->Od.bytes < obytes) {
    s->Od.release();
    if (s->Od.ensure(obytes) != cudaSuccess) return fail(FTLM_ERR_OUT_OF_MEMORY, "O matrices");
  }
  // u.S q_k of all stored vectors (as large as the stored vectors)
  const size_t wbytes = (size_t)d * R * (c64 ? 8 : 16) * M;
  if (s->Ws.bytes < wbytes) {
    s->Ws.release();
    if (s->Ws.ensure(wbytes) != cudaSuccess)
      return fail(FTLM_ERR_OUT_OF_MEMORY, "symmetric run: " + std::to_string(wbytes) + " bytes for u.S of the Lanczos vectors");
  }
  void* W = s->Ws.p;
  InstDesc hd = base_desc(s, c64);
  observable_coefs(s->hs, p->obs_dir, hd.obs);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  CKI(launch_sym_omat(&hd, s->Vs.p, W, R, M, nranges, reinterpret_cast<double*>(s->Wc.p),
                      reinterpret_cast<double*>(s->Od.p), c64, st));
  CK(cudaEventRecord(e1, st));
  std::vector<double> host((size_t)R * M * M * 2);
  CK(cudaMemcpyAsync(host.data(), s->Od.p, obytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float fms = 0.f;
  CK(cudaEventElapsedTime(&fms, e0, e1));
  ms = fms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  Omat.assign((size_t)R * M * M * 2, 0.0);
  for (int r = 0; r < R; ++r)
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        const size_t e = ((size_t)r * M + i) * M + j;
        const double sc = sigma[(size_t)i * R + r] * sigma[(size_t)j * R + r];
        Omat[2 * e] = sc * host[2 * e];
        Omat[2 * e + 1] = sc * host[2 * e + 1];
      }
  return FTLM_OK;
}

ftlm_status run_impl(std::vector<ftlm_system*> sys, const ftlm_run_params* p, ftlm_result* res) {
  ftlm_status vs = validate_params(p, sys);
  if (vs != FTLM_OK) return vs;
  if (!res) return fail(FTLM_ERR_INVALID_ARG, "result is NULL");
  const int c64 = p->dtype == FTLM_C64;
  const int R = p->R, M = p->M, n = (int)sys.size();
  int dev = 0;
  CK(cudaGetDevice(&dev));
  for (auto* s : sys)
    if (s->device != dev) return fail(FTLM_ERR_INVALID_ARG, "system lives on another device");
  const cudaStream_t caller = pick_stream(sys[0], p->stream);
  const cudaStream_t st = sys[0]->own_stream;  // graphs are captured and launched on the first system's stream
  for (auto* s : sys) {
    ftlm_status w = ensure_workspace(s, R, M, c64);
    if (w != FTLM_OK) return w;
  }
  Plan pl;
  ftlm_status ps;
  if (p->reorth) {  // the general row kernel on the row-major block, gather and update in two launches
    Shape gen = default_shape(R, c64);
    gen.explicit_general = true;
    ps = make_plan(sys, R, c64, pl, &gen, false);
    pl.wideV = 0;
  } else {
    ps = make_plan(sys, R, c64, pl, nullptr, true);
  }
  if (ps != FTLM_OK) return ps;
  if (vm_fused_step(pl)) {
    ftlm_status ut = ensure_unit_tables(sys[0], pl.half.K, c64, st);
    if (ut != FTLM_OK) return ut;
  }
  if (pl.half.on && !vm_fused_step(pl)) {  // (the fused vector-major step keeps no H q block)
    ftlm_status hs_ = ensure_hq(sys[0], R, c64, (pl.half.vm && !pl.half.hybrid) ? pl.half.passes : 1);
    if (hs_ != FTLM_OK) return hs_;
  } else if (pl.wideV || (pl.gen_vm && !pl.gvm_cube)) {  // (the cube gather keeps no H q block)
    for (auto* s : sys) {
      ftlm_status hs_ = ensure_hq(s, R, c64, 1);
      if (hs_ != FTLM_OK) return hs_;
    }
  }
  if (p->symmetric || p->reorth) {  // the M Lanczos vectors of every vector
    ftlm_system* s0 = sys[0];
    const size_t vb = (size_t)s0->hs.dim * R * (c64 ? 8 : 16) * M;
    if (s0->Vs.bytes < vb) {
      s0->Vs.release();
      if (s0->Vs.ensure(vb) != cudaSuccess)
        return fail(FTLM_ERR_OUT_OF_MEMORY, std::string(p->symmetric ? "symmetric" : "re-orthogonalised") +
                                                " run: " + std::to_string(vb) + " bytes of Lanczos vectors");
      s0->gen++;
    }
  }
  if (p->reorth) {
    ftlm_system* s0 = sys[0];
    const size_t gb = sizeof(double) * 2 * (size_t)R * M;
    if (s0->Gre.bytes < gb) {
      s0->Gre.release();
      CK(s0->Gre.ensure(gb));
      s0->gen++;
    }
  }
  const std::string key = run_key(sys, p, pl);
  RunCtx* ctx = nullptr;
  size_t h2d = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& c : g_ctx)
      if (c->key == key) ctx = c.get();
  }
  if (!ctx) {
    auto nc = std::make_unique<RunCtx>();
    nc->key = key;
    ftlm_status bs = build_ctx(*nc, sys, p, pl, st);
    if (bs != FTLM_OK) return bs;
    h2d = nc->h2d;
    ctx = nc.get();
    std::lock_guard<std::mutex> lk(g_mu);
    g_ctx.push_back(std::move(nc));
    if (g_ctx.size() > 8) g_ctx.erase(g_ctx.begin());
  }
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaEventRecord(sys[0]->ev_in, caller));  // after the caller's prior work (e.g. a user start block)
  CK(cudaStreamWaitEvent(st, sys[0]->ev_in, 0));
  CK(cudaGraphLaunch(ctx->ex, st));
  CK(cudaEventRecord(sys[0]->ev_out, st));
  CK(cudaStreamWaitEvent(caller, sys[0]->ev_out, 0));  // the caller's later work sees the run complete
  CK(cudaStreamSynchronize(st));
  const auto t1 = std::chrono::steady_clock::now();
  double hv_ms = 0.0, gap_ms = 0.0, dev_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (p->time_kernels && !ctx->ev.empty()) {
    for (int j = 0; j < M; ++j) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ctx->ev[2 + 4 * j], ctx->ev[3 + 4 * j]));
      hv_ms += ms;
      if (j + 1 < M) {
        CK(cudaEventElapsedTime(&ms, ctx->ev[4 + 4 * j], ctx->ev[1 + 4 * (j + 1)]));
        gap_ms += ms;
      }
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[4 * M + 1]));
    dev_ms = ms;
  }
  const size_t per = staged_bytes(R, M);
  for (int k = 0; k < n; ++k) {  // host: eigensolve + sums per instance
    const char* src = ctx->pinned + per * k;
    const double* alpha_d = reinterpret_cast<const double*>(src);  // [M][R]
    const double* beta_d = alpha_d + (size_t)M * R;
    const double* p_d = beta_d + (size_t)M * R;                     // [M][R][2]
    const int* meff = reinterpret_cast<const int*>(src + sizeof(double) * staged_doubles(R, M));
    std::vector<double> al((size_t)R * M), be((size_t)R * M), pp((size_t)R * M * 2);
    for (int r = 0; r < R; ++r)
      for (int j = 0; j < M; ++j) {
        al[(size_t)r * M + j] = alpha_d[(size_t)j * R + r];
        be[(size_t)r * M + j] = beta_d[(size_t)j * R + r];
        pp[((size_t)r * M + j) * 2] = p_d[((size_t)j * R + r) * 2];
        pp[((size_t)r * M + j) * 2 + 1] = p_d[((size_t)j * R + r) * 2 + 1];
      }
    std::vector<int> me(meff, meff + R);
    for (int r = 0; r < R; ++r)
      if (me[r] < 1 || me[r] > M) return fail(FTLM_ERR_NUMERICAL, "start vector of zero norm");
    ftlm_result& out = res[k];
    std::string msg;
    ftlm_status ss = host_sums(R, M, me.data(), al.data(), be.data(), pp.data(), (double)sys[k]->hs.dim,
                               sys[k]->hs.g, p->T, p->nT, &out, msg);
    if (ss != FTLM_OK) return fail(ss, msg);
    if (out.alpha) std::memcpy(out.alpha, al.data(), sizeof(double) * al.size());
    if (out.beta) std::memcpy(out.beta, be.data(), sizeof(double) * be.size());
    if (out.p) std::memcpy(out.p, pp.data(), sizeof(double) * pp.size());
    if (out.M_eff) std::memcpy(out.M_eff, me.data(), sizeof(int) * R);
    out.device_ms = dev_ms;
    out.hv_ms = hv_ms;
    out.gap_ms = gap_ms;
    out.hv_launches = ctx->hv_launches;
    out.kernel_launches = ctx->launches;
    out.h2d_bytes = k == 0 ? h2d : 0;
    out.d2h_bytes = per;
    out.cube_bits = pl.half.on ? pl.half.K : 0;  // (0 also for the vector-major general gather)
    out.passes = pl.half.on ? pl.half.passes : 1;
    out.group_vectors = pl.half.on ? pl.half.Rg : (pl.gen_vm ? pl.gvm_V : R);
    out.tile_rows = pl.half.on ? pl.half.rows_per_tile : (pl.gen_vm ? pl.gvm_rows : pl.sh.rows_per_tile);
    out.grid = pl.half.on ? pl.half.grid : (pl.gen_vm ? pl.gvm_grid : pl.grid);
    out.threads = pl.half.on ? pl.half.threads : (pl.gen_vm ? 256 : pl.sh.threads);
    out.vector_major = plan_vmaj(pl) ? 1 : 0;
    out.site_cube = pl.gen_vm ? pl.gvm_cube : 0;
    out.sym_ms = 0.0;
    if (p->symmetric) {  // Eqs. (E-2-G), (E-2-H)
      const double* sigma_d = p_d + (size_t)M * R * 2;  // [M][R]
      std::vector<double> Omat;
      double sms = 0.0;
      ftlm_status os = symmetric_matrices(sys[k], p, st, sigma_d, Omat, sms);
      if (os != FTLM_OK) return os;
      out.sym_ms = sms;
      if (out.M_B_sym) {
        std::string m2;
        ftlm_status hs2 = host_sums_sym(R, M, me.data(), al.data(), be.data(), Omat.data(), sys[k]->hs.g, p->T,
                                        p->nT, out.M_B_sym, out.M_B_sym_imag, m2);
        if (hs2 != FTLM_OK) return fail(hs2, m2);
      }
      if (out.O_lanczos) std::memcpy(out.O_lanczos, Omat.data(), sizeof(double) * Omat.size());
    }
  }
  return FTLM_OK;
}

// Times candidate launch shapes of the H.v kernel on the system's workspace
// and keeps the fastest for (n, 2s+1, R, dtype, d).
ftlm_status autotune(ftlm_system* s, int R, int c64, cudaStream_t st) {
  ShapeKey key{s->hs.n, s->hs.qmax, R, c64, (long long)s->hs.dim};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_shapes.count(key)) return FTLM_OK;
  }
  std::vector<Shape> cands;
  if (s->hs.all_half && s->hs.n >= 4) {
    std::vector<int> rgs;
    for (int cap : {64, 32, 16}) {
      const int g = largest_divisor_at_most(R, cap);
      if (std::find(rgs.begin(), rgs.end(), g) == rgs.end()) rgs.push_back(g);
    }
    for (int mp : {0, 1})
      for (int K : {3, 4})
        for (int rg : rgs)
          for (int f : {1, 4})  // cubes per thread slot in a row tile
            for (int mb : {2, 3}) {
              if (mp && mb > 1) continue;
              Shape sh = default_shape(R, c64);
              sh.half_K = K;
              sh.Rg = rg;
              sh.half_rows = f;
              sh.half_multipass = mp;
              sh.half_min_blocks = mb;
              if (s->hs.n >= K + 2) cands.push_back(sh);
            }
    for (int mp : {0, 1, 2})  // the vector-major gather (runs only): one pass, ceil((n-5)/K) passes, two passes
      for (int K : {3, 4})
        for (int f : {1, 2, 4, 8})
          for (int mb : {1, 2}) {  // one 512-thread or two 256-thread CTAs per SM
            Shape sh = default_shape(R, c64);
            sh.half_K = K;
            sh.Rg = largest_divisor_at_most(R, 16);
            sh.half_rows = f;
            sh.half_multipass = mp == 1 ? 1 : 0;
            sh.half_hybrid = mp == 2 ? 1 : 0;
            sh.half_min_blocks = mb;
            sh.half_vm = 1;
            if (s->hs.n >= kVmLaneBits + (mp == 2 ? 2 * K : K)) cands.push_back(sh);
          }
  } else {
    for (int thr : {128, 256})
      for (int f : {1, 4}) {
        Shape sh = shape_for(R, c64, thr, f);
        sh.general_vm = 0;
        cands.push_back(sh);
      }
    for (int cube : {8, 4, 0})  // the vector-major general gather (runs only): cube over 8 or 4 vectors, none
      for (int rows : {256, 512, 1024, 2048}) {
        Shape sh = default_shape(R, c64);
        sh.general_vm = 1;
        sh.gvm_rows = rows;
        sh.gvm_cube = cube;
        cands.push_back(sh);
      }
  }
  ftlm_status w = ensure_workspace(s, R, 1, c64);
  if (w != FTLM_OK) return w;
  const size_t vbytes = (size_t)s->hs.dim * (c64 ? 8 : 16);
  CK(cudaMemsetAsync(s->A.p, 0, vbytes * R, st));
  DevBuf vdesc;  // the vector-major candidates: one descriptor per vector, output in Hq (one block per pass)
  DevBuf vtiles; // the vector-major general candidates' tile lists
  if (!s->hs.all_half || s->hs.n >= kVmLaneBits + 3) {
    const int passes = s->hs.all_half ? (s->hs.n - kVmLaneBits + 2) / 3 : 1;  // the most passes a candidate uses
    ftlm_status hq = ensure_hq(s, R, c64, passes);
    if (hq != FTLM_OK) return hq;
    std::vector<InstDesc> h(R, base_desc(s, c64));
    for (int k = 0; k < R; ++k) {
      h[k].x = static_cast<char*>(s->A.p) + vbytes * k;
      h[k].y = static_cast<char*>(s->Hq.p) + vbytes * k;
    }
    CK(vdesc.ensure(sizeof(InstDesc) * R));
    CK(cudaMemcpy(vdesc.p, h.data(), sizeof(InstDesc) * R, cudaMemcpyHostToDevice));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  Shape pick = default_shape(R, c64);
  std::vector<ftlm_system*> one{s};
  for (const Shape& sh : cands) {
    Plan pl;
    if (make_plan(one, R, c64, pl, &sh, sh.half_vm != 0 || sh.general_vm == 1) != FTLM_OK) continue;
    if (sh.half_K > 0 && (!pl.half.on || pl.half.vm != (sh.half_vm != 0))) continue;
    if (sh.general_vm == 1 && (!pl.gen_vm || (sh.gvm_cube > 0 && (!pl.gvm_cube || pl.gvm_V != sh.gvm_cube)))) continue;
    LaunchArgs a = pl.base;
    if (pl.half.vm) {
      a.inst = reinterpret_cast<const InstDesc*>(vdesc.p);
    } else if (pl.gen_vm) {  // R one-vector instances, then the groups' tile list
      std::vector<int> tiles = pl.tile_start;
      tiles.insert(tiles.end(), pl.tile_start_g.begin(), pl.tile_start_g.end());
      CK(cudaStreamSynchronize(st));  // (the previous candidate's launches may read the old list)
      CK(vtiles.ensure(sizeof(int) * tiles.size()));
      CK(cudaMemcpy(vtiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice));
      a.inst = reinterpret_cast<const InstDesc*>(vdesc.p);
      a.tile_start = reinterpret_cast<const int*>(vtiles.p);
    } else {
      a.inline_one = 1;
      a.one = base_desc(s, c64);
      a.one.x = s->A.p;
      a.one.y = s->B.p;
    }
    a.mode = kModeApply;
    for (int it = 0; it < 2; ++it) CKI(launch_plan(pl, a, st));  // warm-up
    CK(cudaEventRecord(e0, st));
    for (int it = 0; it < 5; ++it) CKI(launch_plan(pl, a, st));
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (pl.half.vm && pl.half.passes > 1 && !pl.half.hybrid)  // the step then reads passes - 1 more H q blocks (~6 TB/s)
      ms += 5.0f * (float)((double)(pl.half.passes - 1) * (double)vbytes * R / 6.0e9);
    if (ms < best) {
      best = ms;
      pick = sh;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  vdesc.release();  // (every candidate's launches have completed: each ends with an event wait)
  vtiles.release();
  std::lock_guard<std::mutex> lk(g_mu);
  g_shapes[key] = pick;
  return FTLM_OK;
}

ftlm_status check_block_args(const ftlm_system* s, const void* x, const void* y, int nvec, ftlm_dtype dtype) {
  if (!s) return fail(FTLM_ERR_INVALID_ARG, "system is NULL");
  if (dtype != FTLM_C64 && dtype != FTLM_C128) return fail(FTLM_ERR_INVALID_ARG, "unknown dtype");
  const int c64 = dtype == FTLM_C64;
  if (nvec < 1 || nvec > max_vectors(c64))
    return fail(FTLM_ERR_INVALID_ARG, "nvec must be in 1.." + std::to_string(max_vectors(c64)));
  if (!x || !y) return fail(FTLM_ERR_INVALID_ARG, "vector blocks must not be NULL");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
    return fail(FTLM_ERR_INVALID_ARG, "vector blocks must be 16-byte aligned");
  return FTLM_OK;
}

// The coupling tables and the workspace of a system live on the device that
// was current when it was created; work for it must be enqueued with that
// device current (pointers of one device are not valid on another).
ftlm_status check_device(const ftlm_system* s) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != s->device)
    return fail(FTLM_ERR_INVALID_ARG, "system lives on device " + std::to_string(s->device) + ", current device is " +
                                          std::to_string(dev));
  return FTLM_OK;
}

ftlm_status rows_entry(const ftlm_system* cs, int mode, const double* u, const void* x, void* y, int nvec,
                       ftlm_dtype dtype, void* stream) {
  ftlm_status v = check_block_args(cs, x, y, nvec, dtype);
  if (v != FTLM_OK) return v;
  v = check_device(cs);
  if (v != FTLM_OK) return v;
  const int c64 = dtype == FTLM_C64;
  ftlm_system* s = const_cast<ftlm_system*>(cs);
  const size_t bytes = (size_t)s->hs.dim * nvec * (c64 ? 8 : 16);
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  if (xa < ya + bytes && ya < xa + bytes) return fail(FTLM_ERR_INVALID_ARG, "x and y overlap");
  Plan pl;
  std::vector<ftlm_system*> one{s};
  if (mode == kModeApply && nvec > 1 && !has_shape_override(s, nvec, c64)) {
    // spin-1/2 blocks on the default plan: transpose to vector-major, the runs'
    // gather, transpose back
    Plan vp;
    ftlm_status ps = make_plan(one, nvec, c64, vp, nullptr, true);
    if (ps == FTLM_OK && vp.half.on && vp.half.vm && vp.half.passes == 1 && !vp.half.hybrid) {
      // the system's two transposed blocks are shared by its calls: a call waits
      // for the previous one's kernels (on whatever stream it ran) before reusing them
      std::lock_guard<std::mutex> lk(s->mu);
      const size_t block = (size_t)s->hs.dim * nvec * (c64 ? 8 : 16);
      if (s->Ta.bytes < block || s->Tb.bytes < block) {
        if (s->apply_used) CK(cudaEventSynchronize(s->ev_apply));
        s->Ta.release();
        s->Tb.release();
        CK(s->Ta.ensure(block));
        CK(s->Tb.ensure(block));
        s->apply_used = false;
      }
      cudaStream_t st = pick_stream(s, stream);
      if (s->apply_used) CK(cudaStreamWaitEvent(st, s->ev_apply, 0));
      ftlm_status ut = ensure_unit_tables(s, vp.half.K, c64, st);
      if (ut != FTLM_OK) return ut;
      CKI(launch_to_vector_major(x, s->Ta.p, (long long)s->hs.dim, nvec, c64, st));
      LaunchArgs a = vp.base;
      a.unit_tab = s->ut[c64 ? 1 : 0].p;
      a.inline_one = 1;
      a.one = base_desc(s, c64);
      a.one.x = s->Ta.p;
      a.one.y = s->Tb.p;
      a.vm_stride = (long long)s->hs.dim * (c64 ? 8 : 16);
      a.mode = kModeApply;
      a.gather_alpha = 0;
      CKI(launch_plan(vp, a, st));
      CKI(launch_from_vector_major(s->Tb.p, y, (long long)s->hs.dim, nvec, c64, st));
      CK(cudaEventRecord(s->ev_apply, st));
      s->apply_used = true;
      return FTLM_OK;
    }
  }
  // one vector: the row-major and the vector-major layouts coincide, so H.v may
  // use the vector-major gather
  ftlm_status ps = make_plan(one, nvec, c64, pl, nullptr, mode == kModeApply && nvec == 1);
  if (ps != FTLM_OK) return ps;
  if (pl.half.vm && pl.half.passes > 1) {  // the multi-pass form writes one block per pass: not for a caller's y
    ps = make_plan(one, nvec, c64, pl);
    if (ps != FTLM_OK) return ps;
  }
  LaunchArgs a = pl.base;
  a.inline_one = 1;
  a.one = base_desc(s, c64);
  a.one.x = x;
  a.one.y = y;
  a.mode = mode;
  observable_coefs(s->hs, u, a.one.obs);
  CKI(launch_plan(pl, a, pick_stream(s, stream)));
  return FTLM_OK;
}

// ---- the allocation-free start block ------------------------------------------
//
// Scratch of ftlm_start_block_noalloc: a file-scope device array instead of
// cudaMalloc.  Layout (doubles): [0, 8) arrival counter; then the per-vector
// scalars of a one-step run (alpha, beta, p, sigma, scale, active, M_eff);
// then the per-CTA partial sums [kNoAllocMaxCtas][kNoAllocMaxVectors][kNumPartials].
constexpr int kNoAllocMaxVectors = 64;
constexpr int kNoAllocMaxCtas = 256;
constexpr size_t kNoAllocScalars = 16 * (size_t)kNoAllocMaxVectors;
constexpr size_t kNoAllocDoubles = 8 + kNoAllocScalars + (size_t)kNoAllocMaxCtas * kNoAllocMaxVectors * kNumPartials;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};  // device address of the array, per device

}  // namespace

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------
extern "C" {

ftlm_status ftlm_start_block_noalloc(const ftlm_system* cs, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                                     ftlm_dtype dtype, void* stream) {
  ftlm_status v = check_block_args(cs, out, out, nvec, dtype);
  if (v != FTLM_OK) return v;
  if (nvec > kNoAllocMaxVectors)
    return fail(FTLM_ERR_INVALID_ARG, "ftlm_start_block_noalloc: nvec " + std::to_string(nvec) +
                                          " exceeds the static scratch (at most " +
                                          std::to_string(kNoAllocMaxVectors) + " vectors)");
  const int c64 = dtype == FTLM_C64;
  ftlm_system* s = const_cast<ftlm_system*>(cs);
  std::lock_guard<std::mutex> lk(s->mu);
  v = check_device(s);
  if (v != FTLM_OK) return v;
  const int dev = s->device;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(FTLM_ERR_UNSUPPORTED, "device ordinal too large");
  void* base = nullptr;
  {
    // once per device, with that device current: the host-side name of the
    // array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> l2(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  double* scratch = reinterpret_cast<double*>(base);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  double* scal = scratch + 8;
  double* partials = scal + kNoAllocScalars;
  cudaStream_t st = pick_stream(s, stream);
  Plan pl;
  std::vector<ftlm_system*> one{s};
  ftlm_status ps = make_plan(one, nvec, c64, pl);
  if (ps != FTLM_OK) return ps;
  const int grid = std::min(pl.grid, kNoAllocMaxCtas);
  // the arrival counter must start at zero; everything else is overwritten
  CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  InstDesc h = base_desc(s, c64);
  CKI(launch_start_random(&h, nullptr, nvec, seed, vec_offset, out, c64, st));
  LaunchArgs a = pl.base;
  a.inline_one = 1;
  a.one = h;
  a.one.x = out;
  a.one.y = out;
  a.one.M = 1;
  a.one.sc = scalars_at(scal, nvec, 1);
  a.partials = partials;
  a.counter = counter;
  a.mode = kModeStartNorm;
  CKI(launch_rows(a, c64, grid, pl.sh.threads, pl.smem, st));
  a.mode = kModeScale;
  CKI(launch_rows(a, c64, grid, pl.sh.threads, pl.smem, st));
  return FTLM_OK;
}

ftlm_status ftlm_system_create(int n_sites, const int* two_s, const double* J, const double* d_ion,
                               const double* e_axes, double g, const double B[3], const double* pos,
                               const ftlm_constants* k, ftlm_system** out) {
  if (!out) return fail(FTLM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string msg;
  auto s = std::make_unique<ftlm_system>();
  ftlm_status st = build_host_system(n_sites, two_s, J, d_ion, e_axes, g, B, pos, k, s->hs, msg);
  if (st != FTLM_OK) return fail(st, msg);
  CK(cudaGetDevice(&s->device));
  CK(cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_apply, cudaEventDisableTiming));
  {
    std::lock_guard<std::mutex> lk(g_mu);
    s->id = g_next_id++;
  }
  const HostSystem& hs = s->hs;
  std::vector<float> tf(hs.tab.begin(), hs.tab.end());
  std::vector<long long> stv(hs.stride.begin(), hs.stride.end());
  cudaError_t e = s->tab_d.ensure(hs.tab.size() * sizeof(double));
  if (e == cudaSuccess) e = s->tab_f.ensure(tf.size() * sizeof(float));
  if (e == cudaSuccess) e = s->stride.ensure(stv.size() * sizeof(long long));
  if (e == cudaSuccess) e = s->q.ensure(hs.q.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(s->tab_d.p, hs.tab.data(), hs.tab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->tab_f.p, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->stride.p, stv.data(), stv.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->q.p, hs.q.data(), hs.q.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->tab_d.release();
    s->tab_f.release();
    s->stride.release();
    s->q.release();
    cudaEventDestroy(s->ev_in);
    cudaEventDestroy(s->ev_out);
    cudaEventDestroy(s->ev_apply);
    cudaStreamDestroy(s->own_stream);
    return fail(e == cudaErrorMemoryAllocation ? FTLM_ERR_OUT_OF_MEMORY : FTLM_ERR_CUDA,
                std::string("uploading the coupling tables: ") + cudaGetErrorString(e));
  }
  *out = s.release();
  return FTLM_OK;
}

void ftlm_system_destroy(ftlm_system* s) {
  if (!s) return;
  cudaDeviceSynchronize();  // the system's buffers may be in use on any stream
  purge_ctx_of(s->id);
  for (DevBuf* b : {&s->tab_f, &s->tab_d, &s->stride, &s->q, &s->A, &s->B, &s->U, &s->scal, &s->ep, &s->ecnt,
                    &s->esc, &s->Hq, &s->Vs, &s->Wc, &s->Od, &s->Gre, &s->Ta, &s->Tb, &s->ut[0], &s->ut[1], &s->Ws})
    b->release();
  cudaEventDestroy(s->ev_in);
  cudaEventDestroy(s->ev_out);
  cudaEventDestroy(s->ev_apply);
  cudaStreamDestroy(s->own_stream);
  delete s;
}

uint64_t ftlm_system_dim(const ftlm_system* s) { return s ? s->hs.dim : 0; }

uint64_t ftlm_system_table_bytes(const ftlm_system* s) {
  if (!s) return 0;
  return (uint64_t)s->hs.tab.size() * (sizeof(double) + sizeof(float)) +
         (uint64_t)s->hs.n * (sizeof(long long) + sizeof(int));
}

ftlm_status ftlm_apply_h(const ftlm_system* s, const void* x, void* y, int nvec, ftlm_dtype dtype, void* stream) {
  return rows_entry(s, kModeApply, nullptr, x, y, nvec, dtype, stream);
}

ftlm_status ftlm_apply_sdir(const ftlm_system* s, const double* u, const void* x, void* y, int nvec,
                            ftlm_dtype dtype, void* stream) {
  if (u && !(std::isfinite(u[0]) && std::isfinite(u[1]) && std::isfinite(u[2])))
    return fail(FTLM_ERR_INVALID_ARG, "u must be finite");
  return rows_entry(s, kModeApplyS, u, x, y, nvec, dtype, stream);
}

}  // extern "C"

namespace {

// Normalised start block: plain random vectors, or pairs of time-reversed ones.
ftlm_status start_block_impl(const ftlm_system* cs, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                             ftlm_dtype dtype, void* stream, bool pairs) {
  ftlm_status v = check_block_args(cs, out, out, nvec, dtype);
  if (v != FTLM_OK) return v;
  const int c64 = dtype == FTLM_C64;
  ftlm_system* s = const_cast<ftlm_system*>(cs);
  std::lock_guard<std::mutex> lk(s->mu);
  v = check_device(s);
  if (v != FTLM_OK) return v;
  cudaStream_t st = pick_stream(s, stream);
  Plan pl;
  std::vector<ftlm_system*> one{s};
  ftlm_status ps = make_plan(one, nvec, c64, pl);
  if (ps != FTLM_OK) return ps;
  // scratch owned by the system: per-CTA partials, the arrival counter and sigma_0
  const size_t pbytes = sizeof(double) * (size_t)pl.grid * nvec * kNumPartials;
  if (s->ep.bytes < pbytes) CK(s->ep.ensure(pbytes));
  if (!s->ecnt.p) {
    CK(s->ecnt.ensure(64));
    CK(cudaMemsetAsync(s->ecnt.p, 0, 64, st));
  }
  if (s->esc.bytes < scalar_bytes(nvec, 1)) CK(s->esc.ensure(scalar_bytes(nvec, 1)));
  InstDesc h = base_desc(s, c64);
  if (pairs) CKI(launch_start_pairs(&h, nvec, seed, vec_offset, out, c64, st, 0));
  else CKI(launch_start_random(&h, nullptr, nvec, seed, vec_offset, out, c64, st));
  LaunchArgs a = pl.base;
  a.inline_one = 1;
  a.one = h;
  a.one.x = out;
  a.one.y = out;
  a.one.M = 1;
  a.one.sc = scalars_at(s->esc.p, nvec, 1);
  a.partials = reinterpret_cast<double*>(s->ep.p);
  a.counter = reinterpret_cast<unsigned*>(s->ecnt.p);
  a.mode = kModeStartNorm;
  CKI(launch_rows(a, c64, pl.grid, pl.sh.threads, pl.smem, st));
  a.mode = kModeScale;
  CKI(launch_rows(a, c64, pl.grid, pl.sh.threads, pl.smem, st));
  return FTLM_OK;
}

}  // namespace

extern "C" {

ftlm_status ftlm_start_block(const ftlm_system* cs, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                             ftlm_dtype dtype, void* stream) {
  return start_block_impl(cs, seed, vec_offset, out, nvec, dtype, stream, false);
}

ftlm_status ftlm_start_pairs(const ftlm_system* cs, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                             ftlm_dtype dtype, void* stream) {
  return start_block_impl(cs, seed, vec_offset, out, nvec, dtype, stream, true);
}

ftlm_status ftlm_time_reverse(const ftlm_system* cs, const void* x, void* y, int nvec, ftlm_dtype dtype,
                              void* stream) {
  ftlm_status v = check_block_args(cs, x, y, nvec, dtype);
  if (v != FTLM_OK) return v;
  const int c64 = dtype == FTLM_C64;
  const size_t bytes = (size_t)cs->hs.dim * nvec * (c64 ? 8 : 16);
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  if (xa < ya + bytes && ya < xa + bytes) return fail(FTLM_ERR_INVALID_ARG, "x and y overlap");
  v = check_device(cs);
  if (v != FTLM_OK) return v;
  InstDesc h = base_desc(cs, c64);
  CKI(launch_time_reverse(&h, x, y, nvec, c64, pick_stream(cs, stream)));
  return FTLM_OK;
}

ftlm_status ftlm_run(const ftlm_system* s, const ftlm_run_params* p, ftlm_result* res) {
  ftlm_system* ms = const_cast<ftlm_system*>(s);
  ftlm_status pv = validate_params(p, {ms});  // host-only: before any lock or CUDA call
  if (pv != FTLM_OK) return pv;
  std::lock_guard<std::mutex> lk(ms->mu);
  if (p && p->autotune) {
    ftlm_status vs = validate_params(p, {ms});
    if (vs != FTLM_OK) return vs;
    vs = check_device(ms);
    if (vs != FTLM_OK) return vs;
    ftlm_status a = autotune(ms, p->R, p->dtype == FTLM_C64, pick_stream(ms, p->stream));
    if (a != FTLM_OK) return a;
  }
  return run_impl({ms}, p, res);
}

ftlm_status ftlm_run_batch(int n, const ftlm_system* const* systems, const ftlm_run_params* p,
                           ftlm_result* results) {
  if (n < 1 || !systems || !results) return fail(FTLM_ERR_INVALID_ARG, "empty batch");
  std::vector<ftlm_system*> v;
  for (int k = 0; k < n; ++k) {
    if (!systems[k]) return fail(FTLM_ERR_INVALID_ARG, "system is NULL");
    for (auto* o : v)
      if (o == systems[k]) return fail(FTLM_ERR_INVALID_ARG, "a system appears twice in the batch");
    v.push_back(const_cast<ftlm_system*>(systems[k]));
  }
  std::vector<ftlm_system*> order = v;  // lock in address order
  std::sort(order.begin(), order.end());
  std::vector<std::unique_lock<std::mutex>> locks;
  for (auto* s : order) locks.emplace_back(s->mu);
  if (p && p->autotune) {
    ftlm_status vs = validate_params(p, v);
    if (vs != FTLM_OK) return vs;
    for (auto* s : v) {
      vs = check_device(s);
      if (vs != FTLM_OK) return vs;
    }
    ftlm_system* big = v[0];
    for (auto* s : v)
      if (s->hs.dim > big->hs.dim) big = s;
    ftlm_status a = autotune(big, p->R, p->dtype == FTLM_C64, pick_stream(v[0], p->stream));
    if (a != FTLM_OK) return a;
  }
  return run_impl(v, p, results);
}

ftlm_status ftlm_tune_shape(const ftlm_system* s, int nvec, ftlm_dtype dtype, int cube_bits, int group_vectors,
                            int tile_cubes, int multipass) {
  if (!s) return fail(FTLM_ERR_INVALID_ARG, "system is NULL");
  if (dtype != FTLM_C64 && dtype != FTLM_C128) return fail(FTLM_ERR_INVALID_ARG, "unknown dtype");
  const int c64 = dtype == FTLM_C64;
  if (nvec < 1 || nvec > max_vectors(c64)) return fail(FTLM_ERR_INVALID_ARG, "nvec out of range");
  ShapeKey key{s->hs.n, s->hs.qmax, nvec, c64, (long long)s->hs.dim};
  if (cube_bits < 0) {  // forget the override (and any autotuned shape)
    std::lock_guard<std::mutex> lk(g_mu);
    g_shapes.erase(key);
    return FTLM_OK;
  }
  Shape sh = default_shape(nvec, c64);
  sh.explicit_general = cube_bits == 0 && multipass == 0;
  if (cube_bits == 0 && multipass != 0) {  // the vector-major general gather
    if (multipass != 1) return fail(FTLM_ERR_INVALID_ARG, "multipass must be 0 or 1 with cube_bits 0");
    if (group_vectors < 0 || group_vectors > 8 || nvec % std::max(1, group_vectors) != 0)
      return fail(FTLM_ERR_INVALID_ARG, "group_vectors must be 0 or a group size (4, 8) dividing nvec");
    if (tile_cubes < 1 || tile_cubes > 64) return fail(FTLM_ERR_INVALID_ARG, "tile_cubes must be in 1..64");
    sh.general_vm = 1;
    sh.gvm_cube = group_vectors;
    sh.gvm_rows = 256 * tile_cubes;
  }
  if (cube_bits != 0) {
    if (!s->hs.all_half) return fail(FTLM_ERR_UNSUPPORTED, "register cubes need every site s = 1/2");
    if (cube_bits < 2 || cube_bits > 4 || s->hs.n < cube_bits + 2)
      return fail(FTLM_ERR_INVALID_ARG, "cube_bits must be 2..4 and at most n_sites - 2");
    if (multipass < 0 || multipass > 9) return fail(FTLM_ERR_INVALID_ARG, "multipass must be in 0..9");
    if (multipass >= 8 && (cube_bits < 3 || s->hs.n < kVmLaneBits + 2 * cube_bits))
      return fail(FTLM_ERR_INVALID_ARG, "the two-pass form needs cube_bits 3..4 and n_sites >= 5 + 2 cube_bits");
    if (multipass >= 3 && (cube_bits < 3 || s->hs.n < kVmLaneBits + cube_bits))
      return fail(FTLM_ERR_INVALID_ARG, "the vector-major kernel needs cube_bits 3..4 and n_sites >= 5 + cube_bits");
    if (multipass < 3 && (group_vectors < 1 || group_vectors > nvec || group_vectors > 256))
      return fail(FTLM_ERR_INVALID_ARG, "group_vectors must be in 1..min(nvec, 256)");
    if (tile_cubes < 1 || tile_cubes > 64) return fail(FTLM_ERR_INVALID_ARG, "tile_cubes must be in 1..64");
    sh.half_K = cube_bits;
    sh.Rg = multipass >= 3 ? largest_divisor_at_most(nvec, 16) : group_vectors;  // row-major fallback for apply_h
    sh.half_rows = tile_cubes;
    sh.half_multipass = (multipass == 1 || multipass == 5 || multipass == 7) ? 1 : 0;
    sh.half_hybrid = multipass >= 8 ? 1 : 0;
    // 2 and 4: 3-CTA register budget; 6, 7 and 8: one 512-thread CTA per SM
    sh.half_min_blocks = (multipass == 2 || multipass == 4) ? 3 : ((multipass >= 6 && multipass <= 8) ? 1 : 2);
    sh.half_vm = multipass >= 3 ? 1 : 0;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_shapes[key] = sh;
  return FTLM_OK;
}

ftlm_status ftlm_sums(int R, int M, const int* M_eff, const double* alpha, const double* beta, const double* p,
                      double dim, double g, const double* T, int nT, ftlm_result* res) {
  std::string msg;
  ftlm_status s = host_sums(R, M, M_eff, alpha, beta, p, dim, g, T, nT, res, msg);
  if (s != FTLM_OK) return fail(s, msg);
  return FTLM_OK;
}

}  // extern "C"

struct ftlm_csr {
  int device = 0;
  int c64 = 1;
  long long dim = 0;
  uint64_t nnz = 0;
  DevBuf rp, col, val;
};

extern "C" {

ftlm_status ftlm_csr_create(const ftlm_system* s, ftlm_dtype dtype, ftlm_csr** out) {
  if (!s || !out) return fail(FTLM_ERR_INVALID_ARG, "system or out is NULL");
  if (dtype != FTLM_C64 && dtype != FTLM_C128) return fail(FTLM_ERR_INVALID_ARG, "unknown dtype");
  *out = nullptr;
  const int c64 = dtype == FTLM_C64;
  const long long dim = (long long)s->hs.dim;
  if (dim >= (1ll << 31)) return fail(FTLM_ERR_UNSUPPORTED, "the stored matrix needs dim < 2^31 (32-bit columns)");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != s->device) return fail(FTLM_ERR_INVALID_ARG, "system lives on another device");
  auto m = std::make_unique<ftlm_csr>();
  m->device = dev;
  m->c64 = c64;
  m->dim = dim;
  LaunchArgs a;
  a.inline_one = 1;
  a.one = base_desc(s, c64);
  a.n_inst = 1;
  a.tab_reals = s->hs.lay.total;
  a.max_n = s->hs.n;
  const size_t smem = csr_smem_bytes(a, c64);
  if (smem > 227 * 1024) return fail(FTLM_ERR_UNSUPPORTED, "coupling tables do not fit in shared memory");
  CKI(csr_prepare(std::max<size_t>(smem, 48 * 1024)));
  cudaStream_t st = s->own_stream;
  DevBuf counts;
  if (counts.ensure(sizeof(int) * (size_t)dim) != cudaSuccess || m->rp.ensure(sizeof(long long) * (size_t)(dim + 1)) != cudaSuccess)
    return fail(FTLM_ERR_OUT_OF_MEMORY, "row pointers");
  CKI(launch_csr_count(a, c64, smem, reinterpret_cast<int*>(counts.p), st));
  CKI(csr_scan(reinterpret_cast<const int*>(counts.p), reinterpret_cast<long long*>(m->rp.p), dim, st));
  long long nnz = 0;
  CK(cudaMemcpyAsync(&nnz, reinterpret_cast<long long*>(m->rp.p) + dim, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  counts.release();
  m->nnz = (uint64_t)nnz;
  if (m->col.ensure(sizeof(int) * (size_t)nnz) != cudaSuccess || m->val.ensure((size_t)nnz * (c64 ? 8 : 16)) != cudaSuccess)
    return fail(FTLM_ERR_OUT_OF_MEMORY, "stored matrix of " + std::to_string(nnz) + " elements");
  CKI(launch_csr_fill(a, c64, smem, reinterpret_cast<const long long*>(m->rp.p), reinterpret_cast<int*>(m->col.p),
                      m->val.p, st));
  CK(cudaStreamSynchronize(st));
  *out = m.release();
  return FTLM_OK;
}

uint64_t ftlm_csr_nnz(const ftlm_csr* m) { return m ? m->nnz : 0; }

uint64_t ftlm_csr_bytes(const ftlm_csr* m) {
  return m ? m->rp.bytes + m->col.bytes + m->val.bytes : 0;
}

ftlm_status ftlm_csr_apply(const ftlm_csr* m, const void* x, void* y, int nvec, void* stream) {
  if (!m) return fail(FTLM_ERR_INVALID_ARG, "matrix is NULL");
  if (nvec < 1 || nvec > max_vectors(m->c64))
    return fail(FTLM_ERR_INVALID_ARG, "nvec must be in 1.." + std::to_string(max_vectors(m->c64)));
  if (!x || !y) return fail(FTLM_ERR_INVALID_ARG, "vector blocks must not be NULL");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
    return fail(FTLM_ERR_INVALID_ARG, "vector blocks must be 16-byte aligned");
  const size_t bytes = (size_t)m->dim * nvec * (m->c64 ? 8 : 16);
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  if (xa < ya + bytes && ya < xa + bytes) return fail(FTLM_ERR_INVALID_ARG, "x and y overlap");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != m->device) return fail(FTLM_ERR_INVALID_ARG, "matrix lives on another device");
  CKI(launch_csr_spmm(m->dim, nvec, reinterpret_cast<const long long*>(m->rp.p), reinterpret_cast<const int*>(m->col.p),
                      m->val.p, x, y, m->c64, reinterpret_cast<cudaStream_t>(stream)));
  return FTLM_OK;
}

void ftlm_csr_destroy(ftlm_csr* m) { delete m; }

ftlm_status ftlm_sums_sym(int R, int M, const int* M_eff, const double* alpha, const double* beta,
                          const double* Omat, double g, const double* T, int nT, double* M_B_sym,
                          double* M_B_sym_imag) {
  if (!M_B_sym) return fail(FTLM_ERR_INVALID_ARG, "M_B_sym is NULL");
  for (int t = 0; T && t < nT; ++t)
    if (!(T[t] > 0.0) || !std::isfinite(T[t])) return fail(FTLM_ERR_INVALID_ARG, "temperatures must be > 0");
  std::string msg;
  ftlm_status s = host_sums_sym(R, M, M_eff, alpha, beta, Omat, g, T, nT, M_B_sym, M_B_sym_imag, msg);
  return s == FTLM_OK ? FTLM_OK : fail(s, msg);
}

const char* ftlm_last_error(void) { return g_err.c_str(); }

const char* ftlm_version(void) { return "ftlm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
