// Internal declarations shared by the host driver and the CUDA kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ftlm.h"

namespace ftlm {

constexpr int kMaxSites = 64;
constexpr int kMaxQ = 16;            // 2s + 1 <= 16
constexpr int kNumPartials = 4;      // per vector: alpha (or |w|^2), Re p, Im p, spare
constexpr uint64_t kMaxDim = 1ull << 36;

// Layout of one system's coupling tables, in units of the table's scalar
// type (float for the c64 path, double for c128).  Host and device compute
// addresses from the same struct.
struct TabLayout {
  int n = 0, qmax = 0;
  int off_m = 0;        // [n][qmax]  m = a - s
  int off_up1 = 0;      // [n][qmax]  <a|s+|a-1>   (0 for a = 0)
  int off_dn1 = 0;      // [n][qmax]  <a|s-|a+1>   (0 for a = 2s)
  int off_up2 = 0;      // [n][qmax]  <a|s+ s+|a-2>
  int off_dn2 = 0;      // [n][qmax]  <a|s- s-|a+2>
  int off_iondiag = 0;  // [n][qmax]  diagonal of d_i (s_i.e_i)^2
  int off_zz = 0;       // [n][n]     coefficient of s^z_i s^z_j (i<j, else 0)
  int off_pm = 0;       // [n][n][2]  coefficient of s+_i s-_j (i<j)
  int off_pp = 0;       // [n][n][2]  coefficient of s+_i s+_j (i<j)
  int off_rho = 0;      // [n][n][2]  coefficient of s+_i s^z_j (any i != j; 0 on the diagonal)
  int off_hp = 0;       // [n][2]     coefficient of s+_i from the Zeeman term
  int off_bz = 0;       // [n][2]     single-ion d e_z b: multiplies (s^z s+ + s+ s^z)
  int off_bb = 0;       // [n][2]     single-ion d b^2: multiplies s+ s+
  int off_hz = 0;       // [n]        coefficient of s^z_i from the Zeeman term
  // packed copies for the general row kernel (one 16-byte shared-memory access each)
  int off_site4 = 0;    // [n][qmax][4]  (<a|s+|a-1>, <a|s-|a+1>, m, single-ion diagonal)
  int off_pair4 = 0;    // [n][n][4]     (s+_i s-_j re, im, s+_i s+_j re, im), i < j
  int total = 0;
};

TabLayout make_layout(int n, int qmax);

// Host copy of a validated system.
struct HostSystem {
  int n = 0;
  std::vector<int> two_s, q;
  std::vector<int64_t> stride;
  uint64_t dim = 0;
  int qmax = 0;
  double g = 2.0;
  double B[3] = {0, 0, 0};
  double Bdir[3] = {0, 0, 1};
  TabLayout lay;
  std::vector<double> tab;  // FP64 tables in layout `lay` (u = field direction)
  bool all_half = false;    // every site s = 1/2
  bool real_pm = true;      // every s+ s- coefficient real (true for J + dipolar)
};

// Validates the inputs and fills `hs`.  Returns FTLM_OK or an error with `msg`.
ftlm_status build_host_system(int n, const int* two_s, const double* J, const double* d_ion,
                              const double* e_axes, double g, const double B[3], const double* pos,
                              const ftlm_constants* k, HostSystem& hs, std::string& msg);

// Coefficients (u_z, Re a_u, Im a_u) of the observable u.S, a_u = (u_x - i u_y)/2;
// u = NULL selects the field direction (z when B = 0).
void observable_coefs(const HostSystem& hs, const double* u, double out[3]);

// ---- device-side descriptors ------------------------------------------------

// Per-instance Lanczos scalars in device memory; arrays are [M][ss] (step
// major) where ss is the scalar row stride: the instance's vectors are
// columns 0..R-1 of these arrays (the pointers may be offset into a larger
// [M][R_total] array when every vector of a run is its own instance).
struct DevScalars {
  int ss = 0;                // row stride of alpha, beta, p (complex), sigma
  double* alpha = nullptr;   // [M][R]
  double* beta = nullptr;    // [M][R]   norm after step j
  double* p = nullptr;       // [M][R][2]
  double* sigma = nullptr;   // [M+1][R] scale: v_j = sigma_j q_j
  double* scale = nullptr;   // [R] running max(|alpha|, beta)
  int* active = nullptr;     // [R]
  int* meff = nullptr;       // [R]
};

struct InstDesc {
  const void* tab = nullptr;       // table scalars (float or double)
  const long long* stride = nullptr;  // [n]
  const int* q = nullptr;          // [n]
  long long dim = 0;
  int n = 0;
  int all_half = 0;
  TabLayout lay;
  // vectors of the current launch
  const void* x = nullptr;   // gather source (q_j), [dim][R]
  void* y = nullptr;         // output (or in place w over q_{j-1})
  const void* u = nullptr;   // observable vector u.S v_0, [dim][R] (Lanczos steps)
  const void* hq = nullptr;  // H q_j written by a separate gather launch (kModeEpilogue)
  DevScalars sc;
  double tol = 0.0;          // breakdown tolerance
  int M = 0;
  double obs[3] = {0, 0, 0}; // observable u.S: u_z, Re a_u, Im a_u with a_u = (u_x - i u_y)/2
};

enum KernelMode : int {
  kModeApply = 0,     // y = H x
  kModeLanczos = 1,   // w = sigma_j H q_j - beta_j sigma_{j-1} q_{j-1} (in place in y), partials alpha, p
  kModeUpdate = 2,    // w -= alpha_j sigma_j q_j (in place in y), partials |w|^2, then beta, sigma
  kModeStartNorm = 3, // partials |x|^2, then sigma_0 = 1/|x|
  kModeApplyS = 4,    // y = scale * (u.S) x  (scale = sigma_0 when Lanczos)
  kModeScale = 5,     // y = sigma_0 x (elementwise; y may equal x)
  kModeEpilogue = 6,  // as kModeLanczos with H q_j read from `hq` instead of gathered (elementwise)
  kModeStep = 7,      // the whole step after a gather that produced alpha_j (gather_alpha):
                      // w = sigma_j hq - beta_j sigma_{j-1} q_{j-1} - alpha_j sigma_j q_j (in place in y),
                      // partials |w|^2, p; then p_j, beta, sigma (elementwise)
};

struct LaunchArgs {
  const InstDesc* inst = nullptr;  // device [n_inst]; unused when inline_one
  const int* tile_start = nullptr; // device [n_inst + 1] prefix sum of tiles per instance; unused when inline_one
  InstDesc one;                    // the single instance, passed by value
  int inline_one = 0;              // 1: n_inst == 1 and the descriptor is `one`
  int n_inst = 0;
  int ntiles = 0;
  int rows_per_tile = 0;
  int R = 0;
  int C = 0;            // vector chunks per row = R / V
  int mode = 0;
  int step = 0;         // Lanczos step j
  int first = 0;        // 1 at j = 0 (no beta term)
  double* partials = nullptr;     // [n_inst][grid][R][kNumPartials]
  unsigned* counter = nullptr;    // zeroed; reset by the last block
  int tab_reals = 0;    // max table size over instances
  int max_n = 0;        // max sites over instances
  int use_sigma0 = 0;   // kModeApplyS: multiply by sigma_0
  // spin-1/2 kernel only: vectors are processed in groups of Rg (tile order
  // is group-major so the gathered slice stays in L2)
  int Rg = 0;           // vectors per group
  int nvg = 0;          // number of vector groups = ceil(R / Rg)
  int tiles_per_vg = 0; // row tiles per vector group
  int real_pm = 0;      // every s+ s- coefficient is real (symmetric coupling tensors)
  // pass of the spin-1/2 kernel: the register cube spans bits [cube_lo, cube_lo + K)
  int cube_lo = 0;      // first bit of the cube
  int new_lo = 0;       // cube bits >= new_lo are this pass's own (their single flips and pairs)
  int later_lo = 0;     // bits >= later_lo outside the cube: partners of the mixed pairs
  int first_pass = 1;   // 1: diagonal, and the output is written; 0: the output is accumulated
  int single_pass = 1;  // 1: the single-pass form (cube on the low K bits, all flags implied)
  int min_blocks = 2;   // register budget of the spin-1/2 kernel: 2 or 3 resident CTAs per SM
  // kModeApply of the spin-1/2 kernels: also sum Re<x|y> per vector, and the
  // last CTA sets alpha_j = sigma_j^2 Re<q_j|H q_j> (x = q_j, y = H q_j)
  int gather_alpha = 0;
  // vector-major multi-pass gather: all npass passes in one launch, pass p
  // writing its partial H x to y + p * pass_stride (complex elements)
  int npass = 1;
  long long pass_stride = 0;
  int hybrid = 0;  // npass = 2: cubes on bits [5, 5 + K) and on the top K bits (see hv_vm.cu)
  // kModeStep / kModeEpilogue: H q_j = sum of hq_parts blocks hq + p * hq_stride
  int hq_parts = 1;
  long long hq_stride = 0;
  // kModeUpdate: 1 = leave w as it is (no alpha term) and only take its norm,
  // beta and sigma (after a re-orthogonalisation)
  int update_no_alpha = 0;
  // vector-major gather of a regular block (inline_one): vector k's x and y
  // are one.x and one.y advanced by k * vm_stride bytes
  long long vm_stride = 0;
  // vector-major one-pass gather of a Lanczos step (x = q_j, y = q_{j-1}, u):
  // writes w' = sigma_j H q_j - beta_j sigma_{j-1} q_{j-1} over q_{j-1} and sums
  // Re<q_j|w'> and <q_j|u>; its last CTA sets alpha_j and p_j.  The rest of
  // the step, w = w' - alpha_j sigma_j q_j with |w|^2, is kModeUpdate.
  int fused_step = 0;
  // vector-major one-pass gather: the system's per-unit coefficient tables
  // (launch_vm_unit_tables), or nullptr to build them in the kernel
  const void* unit_tab = nullptr;
};

// Launch shapes chosen per (path, R, dtype); see autotuning in api.cu.
struct Shape {
  int threads = 256;
  int rows_per_tile = 256;
  int ctas_per_sm = 2;
  int half_K = 0;       // > 0: spin-1/2 register-cube kernel with cubes of 2^half_K rows
  int Rg = 0;           // spin-1/2 kernel: vectors per group
  int half_rows = 2;    // spin-1/2 kernel: cubes per thread slot in a row tile
  int half_multipass = 0;  // spin-1/2 kernel: 1 = ceil(N/K) passes whose cubes cover all bits
  int half_min_blocks = 2; // spin-1/2 kernel: register budget of 2 or 3 CTAs per SM
  int half_vm = 0;         // spin-1/2 kernel: 1 = vector-major Lanczos block (ftlm_run only)
  int half_hybrid = 0;     // vector-major: the two-pass form (cubes on bits [5, 5+K) and the top K bits)
  bool explicit_general = false;  // set by the caller: general kernel even for spin-1/2
  int general_vm = -1;     // general kernel in runs: 1 = vector-major gather, 0 = row-major, -1 = by block size
  int gvm_rows = 1024;     // vector-major general gather: rows per tile
  int gvm_cube = -1;       // vector-major general gather: > 0 = register cube of the top site over groups
                           // of that many vectors, 0 = one row a thread, -1 = the cube with the default
                           // group size where a kernel exists for the top site's 2s+1 and R
};

// Kernel launchers (kernels.cu).  `V` is the number of complex values per
// thread (2 for c64, 1 for c128).  Return cudaError_t as int.
int launch_rows(const LaunchArgs& a, int c64, int grid, int threads, size_t smem, void* stream);
// vector_major: the block is R contiguous vectors of dim values (else dim rows of R values)
int launch_start_random(const InstDesc* inst_host, const InstDesc* inst_dev, int R, uint64_t seed,
                        uint64_t vec_offset, void* out, int c64, void* stream, int vector_major = 0);
int launch_start_basis(long long dim, int R, uint64_t basis_offset, void* out, int c64, void* stream,
                       int vector_major = 0);
int launch_to_vector_major(const void* src, void* dst, long long dim, int R, int c64, void* stream);
// the inverse: dst[nu * R + k] = src[k * dim + nu]
int launch_from_vector_major(const void* src, void* dst, long long dim, int R, int c64, void* stream);
// pairs of time-reversed random vectors (unnormalised) and y = Theta x on [d][R]
int launch_start_pairs(const InstDesc* h, int R, uint64_t seed, uint64_t vec_offset, void* out, int c64,
                       void* stream, int vector_major);
int launch_time_reverse(const InstDesc* h, const void* x, void* y, int R, int c64, void* stream);
int launch_copy_block(const void* src, void* dst, size_t bytes, void* stream);
size_t rows_smem_bytes(const LaunchArgs& a, int c64, int threads, int Vmax = 0);
int launch_rows_wide(const LaunchArgs& a, int V, int grid, int threads, size_t smem, void* stream);
int prepare_rows_kernels(size_t smem);
// CTAs per SM of the Lanczos-mode row kernel, or of the wide H.v kernel when wideV is 4 or 8
int rows_max_ctas_per_sm(int c64, int threads, size_t smem, int wideV);
// vector-major general H.v: V vectors a thread (c64: 1, 2, 4, 8; c128: 1, 2, 4)
int rows_vm_supported(int V, int c64);
int prepare_rows_vm(int V, int c64, size_t smem);
int rows_vm_ctas_per_sm(int V, int c64, int threads, size_t smem);
int launch_rows_vm(const LaunchArgs& a, int V, int c64, int grid, int threads, size_t smem, void* stream);
// The vector-major general H.v with a register cube of the top site's Q = 2s+1
// rows (hv_cube.cu), over groups of cube_vectors(Q, c64) vectors (0: no
// kernel for this Q; want > 0 asks for that group size); tiles are ranges of
// bases (rows with top digit 0).
int cube_vectors(int Q, int c64, int want = 0);
int prepare_cube(int Q, int V, int c64, size_t smem);
// shared memory of rows_vm_kernel and cube_gather_kernel (no reduction space)
size_t gather_smem_bytes(const LaunchArgs& a, int c64, int threads);
int cube_ctas_per_sm(int Q, int V, int c64, int threads, size_t smem);
int launch_cube(const LaunchArgs& a, int Q, int V, int c64, int grid, int threads, size_t smem, void* stream);
int device_sm_count();
long long device_l2_bytes();

// Spin-1/2 register-cube kernel (hv_half.cu): modes kModeApply and kModeLanczos
// of a single instance with every site s = 1/2.
int launch_half(const LaunchArgs& a, int K, int c64, int grid, int threads, size_t smem, void* stream);
size_t half_smem_bytes(int n, int K, int rows_per_tile, int threads);
int prepare_half_kernels(size_t smem);
int half_max_ctas_per_sm(int K, int c64, int threads, size_t smem, int min_blocks, bool multipass, int R);

// Vector-major spin-1/2 kernel (hv_vm.cu): mode kModeApply over R instances,
// one per vector, all of one system; K = 3 or 4.  a.single_pass = 1: one pass
// (a.tiles_per_vg tiles per vector); 0: a.npass passes in the same launch
// (a.tiles_per_vg tiles per vector and pass, outputs a.pass_stride apart).
int launch_vm(const LaunchArgs& a, int K, int min_blocks, int c64, int grid, int threads, size_t smem, void* stream);
size_t vm_smem_bytes(int n, int K, int threads, int npass, int c64);
int set_vm_carveout(int K, int c64, bool multipass, int min_blocks, size_t smem, int ctas);
int prepare_vm_kernels(size_t smem);
int vm_max_ctas_per_sm(int K, int min_blocks, int c64, int threads, size_t smem, bool multipass);
// per-unit coefficient tables of the one-pass form: stride reals a unit,
// d >> (5 + K) units, computed from the FP64 coupling tables
int vm_unit_table_stride(int n, int K);
int launch_vm_unit_tables(const double* tab_d, const TabLayout& L, int n, int K, long long nunits, void* out, int c64,
                          void* stream);
// kModeStep / kModeStartNorm over the same one-vector instances (256 threads)
int launch_vm_stream(const LaunchArgs& a, int c64, int grid, void* stream);
constexpr int kVmLaneBits = 5;  // rows per warp-wide load: 2^5

// Full re-orthogonalisation pass (reorth.cu): w_r -= sum_{k<=j} sigma_k^2 <q_k|w_r> q_k
// for the R vectors of a row-major block w [dim][R], against the stored
// vector-major q_k (Vs [M][R][dim]); G is [R][M] complex FP64 scratch, sigma [M+1][R].
int launch_reorth_pass(const void* Vs, void* w, long long dim, int R, int j, int M, double* G, const double* sigma,
                       int c64, void* stream);

// Symmetric estimator (sym.cu): G[r][i][j] = <q_i|u.S q_j> over the stored
// vector-major Lanczos vectors Vs ([M][R][dim]) of every vector r, complex
// FP64 [R][M][M]; Gp holds sym_partial_doubles(R, M, nranges) doubles.
int sym_ranges(long long dim, int R, int M);
size_t sym_partial_doubles(int R, int M, int nranges);
// W: space for (u.S) q_k of every stored vector (the size of Vs), formed
// first and then loaded by the contraction.
int launch_sym_omat(const InstDesc* h, const void* Vs, void* W, int R, int M, int nranges, double* Gp, double* G,
                    int c64, void* stream);

// Stored-matrix comparison path (csr.cu): count, scan, fill, multiply.
size_t csr_smem_bytes(const LaunchArgs& a, int c64);
int csr_prepare(size_t smem);
int launch_csr_count(const LaunchArgs& a, int c64, size_t smem, int* counts, void* stream);
int launch_csr_fill(const LaunchArgs& a, int c64, size_t smem, const long long* rp, int* col, void* val,
                    void* stream);
int csr_scan(const int* counts, long long* rp, long long dim, void* stream);
int launch_csr_spmm(long long dim, int R, const long long* rp, const int* col, const void* val, const void* x,
                    void* y, int c64, void* stream);

// Host tridiagonal eigensolver + sums (tridiag.cpp); host_sums_sym: the
// symmetric estimator of M_B from the matrices O_ij = <v_i|u.S|v_j>.
ftlm_status host_sums(int R, int M, const int* M_eff, const double* alpha, const double* beta, const double* p,
                      double dim, double g, const double* T, int nT, ftlm_result* res, std::string& msg);
ftlm_status host_sums_sym(int R, int M, const int* M_eff, const double* alpha, const double* beta,
                          const double* Omat, double g, const double* T, int nT, double* MB_sym, double* MB_sym_imag,
                          std::string& msg);

}  // namespace ftlm
