/*
 * ftlm.h -- C ABI of the GB300 finite-temperature Lanczos (FTLM) library.
 *
 * The library evaluates, on one GPU, the hot path of FTLM for anisotropic
 * spin Hamiltonians (arxiv 2607.25585, Schnack): the matrix-free complex
 * H.v over the full product basis, driven by the three-term Lanczos
 * recurrence from random vectors, and the <v_j|O|r> projections that the
 * FTLM estimators need for Z, E, C and M_B.
 *
 * Conventions shared by every call:
 *  - Units: energies and temperatures in Kelvin (k_B = 1), fields in Tesla,
 *    distances in Angstrom.  C is returned in units of k_B per system, M_B in
 *    units of mu_B per system.
 *  - Basis: the (2s_0+1) x ... x (2s_{n-1}+1) product basis of S^z
 *    eigenstates.  Basis index mu = sum_i a_i * prod_{k<i} (2 s_k + 1), with
 *    site 0 the least significant digit and digit a_i = m_i + s_i in
 *    [0, 2 s_i].  This ordering is part of the ABI because vectors are.
 *  - Vector blocks: row-major [dim][nvec], the nvec vectors of one basis
 *    state contiguous, each complex number interleaved (re, im).  FTLM_C64
 *    is 8 bytes per element (two floats), FTLM_C128 16 bytes (two doubles).
 *    Device blocks must be 16-byte aligned.
 *  - Ownership: every pointer passed in stays owned by the caller; inputs are
 *    copied before the call returns (asynchronous device calls read and write
 *    the caller's device buffers until the stream reaches that point).
 *    Objects returned through out-pointers are owned by the library and are
 *    released with the matching destroy call.
 *  - Errors: every call returns an ftlm_status; on failure nothing is
 *    written to outputs that the call owns, and ftlm_last_error() returns a
 *    message (thread-local, valid until the next call on the same thread).
 *    No exception, abort() or exit() crosses this interface.
 *  - Streams are cudaStream_t passed as void*.  The asynchronous calls
 *    (apply_h, apply_sdir, start_block) enqueue their kernels on that stream;
 *    NULL is the CUDA default stream.  ftlm_run / ftlm_run_batch launch their
 *    captured graph on a stream of their own, ordered after the work already
 *    enqueued on the given stream and before any work enqueued there later,
 *    and return when the results are on the host.
 */
#ifndef FTLM_H
#define FTLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FTLM_OK = 0,
  FTLM_ERR_INVALID_ARG = 1,   /* an argument is out of range or inconsistent */
  FTLM_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
  FTLM_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the code) */
  FTLM_ERR_TIMEOUT = 4,       /* reserved: a bounded device wait gave up */
  FTLM_ERR_UNSUPPORTED = 5,   /* valid request outside what the library supports */
  FTLM_ERR_NUMERICAL = 6      /* NaN/Inf in the Lanczos scalars or the eigensolver */
} ftlm_status;

typedef enum {
  FTLM_C128 = 0, /* complex128 vectors, FP64 matvec ("plain" path) */
  FTLM_C64 = 1   /* complex64 vectors, FP32 matvec with FP32 accumulation;
                    FP64 Lanczos scalars, eigensolve and Boltzmann sums */
} ftlm_dtype;

typedef enum {
  FTLM_START_RANDOM = 0, /* Gaussian random vectors, Eq. (2) */
  FTLM_START_BASIS = 1,  /* basis vectors |basis_offset + k>, k = 0..R-1 */
  FTLM_START_USER = 2,   /* caller's device block [dim][R] of the run's dtype */
  FTLM_START_PAIRS = 3   /* pairs of time-reversed random vectors (ftlm_start_pairs) */
} ftlm_start_mode;

/* Physical constants used by Eq. (3); NULL selects the defaults
 * mu_B = 0.6717 K/T and C_dip = mu0 mu_B^2 / (4 pi k_B) = 0.6228 K A^3. */
typedef struct {
  double mu_B;  /* Bohr magneton, K/T */
  double C_dip; /* dipolar prefactor, K Angstrom^3 (multiplied by g^2 / r^3) */
} ftlm_constants;

typedef struct ftlm_system ftlm_system; /* opaque, library-owned */

/*
 * ftlm_system_create -- the spin Hamiltonian of Eq. (3) (Sec. II.A):
 *   H = 2 sum_{i<j} J_ij s_i.s_j + sum_i d_i (s_i.e_i)^2 + mu_B g B.sum_i s_i
 *       + C_dip sum_{i<j} g^2 / r_ij^3 (s_i.s_j - 3 (s_i.e_ij)(e_ij.s_j)),
 * on the product basis of dimension d = prod_i (2 s_i + 1) (Sec. II.A).
 *
 *  n_sites  number of spins, 1..64; d must not exceed 2^36.
 *  two_s    [n_sites] host, 2 s_i, each 1..15.
 *  J        [n_sites * n_sites] host, row-major, Kelvin; only the strict
 *           upper triangle J[i*n+j], i<j, is read.  NULL = no exchange.
 *  d_ion    [n_sites] host, Kelvin, or NULL (no single-ion term).
 *  e_axes   [n_sites * 3] host, single-ion axes, normalised by the library;
 *           a zero axis is allowed only where d_ion is 0.  NULL iff d_ion is NULL.
 *  g        g factor (Zeeman uses g, the dipolar term g^2).
 *  B        [3] host, field in Tesla.
 *  pos      [n_sites * 3] host, positions in Angstrom, or NULL: no dipolar
 *           term.  Coincident positions are rejected.
 *  k        constants, or NULL for the defaults.
 *  out      receives the system; release with ftlm_system_destroy.
 * Validation happens on the host before any CUDA call, so invalid arguments
 * are reported without touching the GPU.  The coupling tables are uploaded
 * to the current CUDA device.
 */
ftlm_status ftlm_system_create(int n_sites, const int* two_s, const double* J, const double* d_ion,
                               const double* e_axes, double g, const double B[3], const double* pos,
                               const ftlm_constants* k, ftlm_system** out);

void ftlm_system_destroy(ftlm_system* sys); /* NULL is a no-op; waits for the system's work */

uint64_t ftlm_system_dim(const ftlm_system* sys); /* d, or 0 for NULL */

/* Bytes that ftlm_system_create copied from the host to the device (the
 * coupling tables in FP32 and FP64, site strides and radices); 0 for NULL. */
uint64_t ftlm_system_table_bytes(const ftlm_system* sys);

/*
 * ftlm_apply_h -- y = H x for a block of nvec vectors, matrix-free (the
 * matrix-vector product that Sec. II.C calls the heart of every Lanczos
 * procedure), evaluated row by row on the GPU from coupling tables: each
 * output row gathers its own terms, so there are no atomics and the result
 * is bitwise reproducible.
 *  x, y   device blocks [dim][nvec] of dtype; must not overlap.
 *  nvec   1..512 (c64) or 1..256 (c128).
 *  stream cudaStream_t or NULL.
 * Asynchronous: returns after enqueueing.
 */
ftlm_status ftlm_apply_h(const ftlm_system* sys, const void* x, void* y, int nvec, ftlm_dtype dtype,
                         void* stream);

/*
 * ftlm_apply_sdir -- y = (u . S) x with S = sum_i s_i, the one-body
 * observable whose projections <v_j|O|r> enter the numerator of Eq. (4).
 *  u      [3] host direction (normalised by the library); NULL = the field
 *         direction B/|B| (z when B = 0).
 * Same block, alignment and stream rules as ftlm_apply_h.
 */
ftlm_status ftlm_apply_sdir(const ftlm_system* sys, const double* u, const void* x, void* y, int nvec,
                            ftlm_dtype dtype, void* stream);

/*
 * ftlm_start_block -- the random start vectors of Eq. (2): out[nu][k] is
 * component nu of random vector number vec_offset + k, with real and
 * imaginary parts independent N(0,1) (Philox4x32-10 keyed by seed, counter
 * (nu, vec_offset + k), Box-Muller in FP64), then each vector normalised to
 * 1 in FP64 (rounded to the dtype afterwards).
 *  out    device block [dim][nvec] of dtype.
 * Asynchronous.  The same (seed, vector number) gives the same vector for
 * any nvec, offset or dtype (up to the final rounding).
 */
ftlm_status ftlm_start_block(const ftlm_system* sys, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                             ftlm_dtype dtype, void* stream);

/*
 * ftlm_time_reverse -- y = Theta x for every column of a block, with Theta =
 * exp(-i pi S^y) K the time-reversal operator (Sec. II.B: the symmetry behind
 * the pairs of mutually time-reversed random vectors): on one site
 * exp(-i pi s^y)|s,m> = (-1)^(s-m)|s,-m>, K conjugates the coefficients, so
 *   y[nu][k] = (-1)^(sum_i a_i(nu)) conj(x[dim - 1 - nu][k])
 * (the digit map a_i -> 2 s_i - a_i reverses the basis index).
 *  x, y   device blocks [dim][nvec] of dtype, 16-byte aligned, not
 *         overlapping (FTLM_ERR_INVALID_ARG otherwise).
 * Asynchronous on stream (NULL = the default stream).
 */
ftlm_status ftlm_time_reverse(const ftlm_system* sys, const void* x, void* y, int nvec, ftlm_dtype dtype,
                              void* stream);

/*
 * ftlm_start_pairs -- start vectors in pairs of mutually time-reversed random
 * vectors (Sec. II.B; tau = 1 in Sec. III): global vector number
 * v = vec_offset + k is random vector v / 2 of ftlm_start_block (same seed)
 * when v is even, and Theta applied to it when v is odd, each normalised to 1.
 * Arguments, layout and stream behaviour as ftlm_start_block; ftlm_run's
 * FTLM_START_PAIRS generates the same vectors.
 */
ftlm_status ftlm_start_pairs(const ftlm_system* sys, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                             ftlm_dtype dtype, void* stream);

/*
 * ftlm_start_block_noalloc -- the same normalised Gaussian start block as
 * ftlm_start_block, for callers that cannot allocate device memory.  Such
 * callers include code running inside a memory budget that someone else
 * owns, or a host that may not call cudaMalloc / cudaFree at that point.
 * This call performs no device allocation and no free, and calls no
 * allocating library routine.  The paper has no counterpart: it is a
 * property of this library's interface, not of the method.
 *
 * Its scratch (per-CTA partial sums of the vector norms, an arrival counter
 * and the per-vector scales) is a file-scope device array of 532,544 bytes
 * that every GPU which loads the library holds until the process exits.
 *  nvec   1..64: larger blocks are rejected with FTLM_ERR_INVALID_ARG
 *         (use ftlm_start_block, which allocates).
 *  The first call on a device looks up the array's device address for that
 *  device (a CUDA runtime query, not an allocation); make that first call
 *  before any stream capture.
 *  All calls on a device share the one array, and it keeps the last call's
 *  contents.  Calls whose GPU work overlaps (concurrent streams, or several
 *  host threads) race on it and give wrong results; order them on one
 *  stream or synchronise between them.
 * Arguments, layout, alignment and stream behaviour as ftlm_start_block.
 */
ftlm_status ftlm_start_block_noalloc(const ftlm_system* sys, uint64_t seed, uint64_t vec_offset, void* out, int nvec,
                                     ftlm_dtype dtype, void* stream);

typedef struct {
  int R;                 /* random vectors (block width), >= 1 */
  int M;                 /* Lanczos steps N_L per vector, >= 1 */
  uint64_t seed;         /* key of the random stream */
  uint64_t vec_offset;   /* global number of the first vector (sharding) */
  ftlm_dtype dtype;      /* FTLM_C64 batched mixed precision, FTLM_C128 plain FP64 */
  int start;             /* ftlm_start_mode */
  uint64_t basis_offset; /* FTLM_START_BASIS: first basis state */
  const void* user_start;/* FTLM_START_USER: device block [dim][R] of dtype */
  const double* T;       /* [nT] host temperatures in K, > 0 */
  int nT;
  const double* obs_dir; /* [3] host direction u of the observable u.S; NULL = B/|B| (z if B = 0) */
  double breakdown_tol;  /* 0 = default (1e-12 for c128, 1e-6 for c64), relative to max(|alpha|, beta) */
  int autotune;          /* 1 = time launch shapes on first use and keep the fastest */
  int time_kernels;      /* 1 = record device time of every H.v launch into the result */
  void* stream;          /* cudaStream_t the run is ordered with; NULL = default stream */
  int symmetric;         /* 1 = also the symmetric estimator of M_B (sFTLM, Eqs. E-2-G/H):
                            keeps all M Lanczos vectors on the device (M x R x dim values of
                            dtype) and as many for u.S of them, forms O_ij = <v_i|u.S|v_j>
                            per vector; one system only */
  int reorth;            /* 0 = none (the three-term recurrence of Sec. II.C, two predecessor
                            vectors: the hot path).  1 = full re-orthogonalisation, the optional
                            step of Sec. II.C: after w = H v_j - alpha_j v_j - beta_j v_{j-1},
                            w -= sum_{k<=j} v_k <v_k|w> is applied twice before beta_{j+1} = |w|.
                            Keeps all M Lanczos vectors on the device (M x R x dim values of
                            dtype, as symmetric), runs the general row kernel, and moves
                            O(M^2 R dim) bytes per run: meant for small dim.  ftlm_run only
                            (ftlm_run_batch returns FTLM_ERR_UNSUPPORTED). */
} ftlm_run_params;

typedef struct {
  /* caller-allocated host outputs, length nT (any may be NULL) */
  double* lnZ;      /* ln Z (Eq. 5); Z itself overflows at low T */
  double* E;        /* internal energy, K */
  double* C;        /* heat capacity, k_B */
  double* M_B;      /* -g <u.S>, mu_B (Eq. 4 with O = u.S) */
  double* M_B_imag; /* imaginary part of the FTLM numerator, a diagnostic */
  /* optional caller-allocated per-vector data ([R][M] row-major; may be NULL) */
  double* alpha;    /* Lanczos diagonal */
  double* beta;     /* beta[r*M + j] = norm after step j (T[j][j+1] for j < M_eff-1) */
  double* p;        /* [R][M][2] complex <v_j|u.S v_0> */
  int* M_eff;       /* [R] Krylov dimension reached (< M after a breakdown) */
  /* filled by the library */
  double E0;              /* lowest Ritz value over all vectors */
  double device_ms;       /* device time of the Lanczos block (start block to last step) */
  double hv_ms;           /* summed device time of the H.v launches (time_kernels = 1) */
  int hv_launches;        /* H.v launches in the run */
  int kernel_launches;    /* all kernel launches in the run */
  uint64_t h2d_bytes;     /* host-to-device bytes copied by the run */
  uint64_t d2h_bytes;     /* device-to-host bytes copied by the run */
  /* launch shape of the H.v launches (see ftlm_tune_shape) */
  int cube_bits;          /* 0: general row kernel; 2..4: spin-1/2 register cubes */
  int passes;             /* launches per H.v (spin-1/2 multi-pass form: ceil(n / cube_bits)) */
  int group_vectors;      /* vectors processed together (register-cube kernels, general vector-major gathers) */
  int tile_rows;          /* rows per tile */
  int grid;               /* CTAs per H.v launch */
  int threads;            /* threads per CTA */
  int vector_major;       /* 1: the run kept each Lanczos vector contiguous (spin-1/2 multipass
                             3..9; other spins with cube_bits 0, multipass 1, or the default plan
                             where the top site's register cube applies or the block fits L2) */
  /* symmetric runs (params.symmetric = 1); caller-allocated, may be NULL */
  double* M_B_sym;        /* [nT] sFTLM: -g sum_r <r|e^{-bH/2} u.S e^{-bH/2}|r> / sum_r <r|e^{-bH}|r>,
                             Eq. (E-2-G) with (E-2-H), shifted by E0 */
  double* M_B_sym_imag;   /* [nT] imaginary part of that numerator, a diagnostic */
  double* O_lanczos;      /* [R][M][M][2] complex O_ij = <v_i|u.S|v_j> (row-major; zero beyond M_eff) */
  double sym_ms;          /* device time of forming O (after the Lanczos run) */
  double gap_ms;          /* time_kernels = 1: summed device time between the end of one Lanczos
                             step's last launch and the start of the next step's first launch
                             (the graph's launch gaps; M - 1 of them) */
  int site_cube;          /* general vector-major H.v: the 2s+1 rows of the top site each thread
                             holds as a register cube (0: one row a thread) */
} ftlm_result;

/*
 * ftlm_run -- plain FTLM, Eqs. (4) and (5) with Gamma = 1 (no symmetry
 * sectors): R start vectors, M Lanczos steps each (three-term recurrence,
 * two predecessor vectors, no re-orthogonalisation; Sec. II.C), the
 * tridiagonal eigenproblem of every vector in FP64, and the Boltzmann sums
 * shifted by the lowest Ritz value E0:
 *   Z' = (d/R) sum_r sum_n |U_0n|^2 e^{-beta (eps_n - E0)},  ln Z = ln Z' - beta E0,
 *   E, C from the same weights, M_B = -g Re[sum e^{-beta(eps-E0)} U_0n sum_j U_jn conj(p_j)] / Z'.
 * All R vectors run as one device block; the M steps are captured in one
 * CUDA graph.  The block is vector-major (each vector contiguous) for
 * spin-1/2 systems and, for other spins, where the general gather can hold
 * the top site's 2s+1 rows as a register cube or the block fits L2; the
 * launch shape is reported in the result (cube_bits, site_cube,
 * vector_major, ...).  Blocks until the results are on the host.
 */
ftlm_status ftlm_run(const ftlm_system* sys, const ftlm_run_params* p, ftlm_result* res);

/*
 * ftlm_run_batch -- ftlm_run for n systems of different dimension at once
 * (e.g. chain lengths x field orientations): one graph, each step one H.v
 * launch and one update launch that cover every instance.  All systems use
 * the same params (R, M, dtype, seed, T grid); results[k] belongs to
 * systems[k].  Blocks until all results are on the host.
 */
ftlm_status ftlm_run_batch(int n, const ftlm_system* const* systems, const ftlm_run_params* p,
                           ftlm_result* results);

/*
 * ftlm_sums -- the host half of Eqs. (4)-(5) on its own: given tridiagonal
 * data of R vectors (as returned in ftlm_result, [R][M] row-major) computes
 * E0, ln Z, E, C, M_B and M_B_imag.  Used to merge vectors run on several
 * processes: gather alpha, beta, p, M_eff from all of them and call this
 * once.  Host-only: needs no GPU.  The R tridiagonal eigenproblems and the
 * temperatures are spread over up to min(R, hardware threads, 32) host
 * threads created and joined inside the call; the result does not depend on
 * their number (each sum runs in a fixed order).  ftlm_run, ftlm_run_batch
 * and ftlm_sums_sym do the same for their host part.
 *  dim  Hilbert-space dimension d; g  g factor.
 */
ftlm_status ftlm_sums(int R, int M, const int* M_eff, const double* alpha, const double* beta, const double* p,
                      double dim, double g, const double* T, int nT, ftlm_result* res);

/*
 * Stored-matrix comparison path.  The paper keeps its Hamiltonian stripes
 * stored on the GPUs in coordinate form, with the elements of one row handled
 * by one thread (Sec. II.C, Table I); ftlm_csr is that matrix in compressed-row
 * form on one device, so that the matrix-free ftlm_apply_h can be measured
 * against it.
 *
 * ftlm_csr_create -- assembles H (Eq. 3) on the current device: the elements
 * of every row as the matrix-free gather enumerates them (diagonal first),
 * exact zeros dropped; row pointers int64 [dim + 1], columns int32 (dim must
 * be below 2^31, else FTLM_ERR_UNSUPPORTED), values complex of dtype.
 * Memory: 8 (dim + 1) + nnz (4 + 8 or 16) bytes (FTLM_ERR_OUT_OF_MEMORY if it
 * does not fit).  Blocks until assembled.  The matrix does not refer to sys
 * afterwards.
 */
typedef struct ftlm_csr ftlm_csr;
ftlm_status ftlm_csr_create(const ftlm_system* sys, ftlm_dtype dtype, ftlm_csr** out);
uint64_t ftlm_csr_nnz(const ftlm_csr* m);    /* stored elements; 0 for NULL */
uint64_t ftlm_csr_bytes(const ftlm_csr* m);  /* device bytes held; 0 for NULL */
/*
 * ftlm_csr_apply -- y = H x with the stored matrix; x, y device blocks
 * [dim][nvec] of the matrix's dtype, 16-byte aligned, not overlapping; nvec
 * as for ftlm_apply_h.  Asynchronous on stream (NULL = default stream).
 */
ftlm_status ftlm_csr_apply(const ftlm_csr* m, const void* x, void* y, int nvec, void* stream);
void ftlm_csr_destroy(ftlm_csr* m);

/*
 * ftlm_sums_sym -- the host half of the symmetric estimator, Eqs. (E-2-G)
 * and (E-2-H), on its own: from the tridiagonal data and the matrices
 * O_ij = <v_i|u.S|v_j> of R runs (as returned in ftlm_result.O_lanczos),
 * M_B_sym[t] and M_B_sym_imag[t] (may be NULL).  E0 is the lowest Ritz
 * value over the R runs, as in ftlm_sums, so vectors run on several
 * processes merge by concatenation.  Host-only: needs no GPU.
 *  Omat  [R][M][M][2] complex, row-major per run.
 */
ftlm_status ftlm_sums_sym(int R, int M, const int* M_eff, const double* alpha, const double* beta,
                          const double* Omat, double g, const double* T, int nT, double* M_B_sym,
                          double* M_B_sym_imag);

/*
 * ftlm_tune_shape -- overrides the launch shape that ftlm_apply_h, ftlm_run
 * and the autotuner use for this system with nvec vectors of dtype (all
 * systems with the same site count, spin values and dimension share it).
 * The default and the autotuner pick these themselves; this call exists for
 * reproducible experiments and tests.
 *  cube_bits      -1: drop the override (back to the default / autotuned
 *                 shape).  0: the general mixed-radix kernel, on the row-major
 *                 block (multipass 0) or, in ftlm_run and ftlm_run_batch, on
 *                 the vector-major block (multipass 1; group_vectors = the
 *                 vectors of one register cube of the top site's 2s+1 rows,
 *                 4 or 8, or 0 for one row a thread; tile_cubes = rows, or
 *                 bases of the cube, per tile in units of 256).  2..4: (every site
 *                 s = 1/2 only) the register-cube kernel in which each thread
 *                 owns 2^cube_bits consecutive rows of one vector.
 *  group_vectors  register-cube kernel: vectors processed together (the
 *                 gathered slice of the block is d * group_vectors elements),
 *                 1..min(nvec, 256).
 *  tile_cubes     register-cube kernel: cubes per thread slot in a row tile, 1..64.
 *  multipass      register-cube kernel: 0 = one launch whose cube is the low
 *                 cube_bits bits; 2 = the same with the register budget of
 *                 three resident CTAs per SM; 1 = ceil(n / cube_bits) launches whose cubes
 *                 cover all bits, so every pair is a cube or cube-neighbour
 *                 pair of one launch (fewer gathered loads, the output is
 *                 re-read by every launch after the first).
 *                 3 = (ftlm_run only; cube_bits 3 or 4, n_sites >= 5 + cube_bits)
 *                 vector-major Lanczos block: each of the R vectors is
 *                 contiguous, the 32 lanes of a warp own 32 consecutive rows
 *                 and each thread a cube along bits [5, 5 + cube_bits), so a
 *                 vector's gathered slice is d elements; 4 = the same with the
 *                 three-CTA register budget; 5 = vector-major in
 *                 ceil((n - 5) / cube_bits) launches whose cubes cover bits
 *                 [5, n), so that every pair is a cube, mixed or lane-lane
 *                 pair of one launch (one output block per pass, summed
 *                 by the step); 6 / 7 = 3 / 5 with one 512-thread CTA per
 *                 SM instead of two of 256; 8 / 9 = vector-major in two
 *                 passes (cubes on bits [5, 5 + cube_bits) and on the top
 *                 cube_bits bits; n_sites >= 5 + 2 cube_bits) with one
 *                 512-thread / two 256-thread CTAs per SM.  group_vectors is ignored and
 *                 tile_cubes counts slabs of 2^(5 + cube_bits) rows per warp.
 *                 ftlm_apply_h on row-major blocks uses the row-major
 *                 register-cube kernel for these shapes.
 * Host-only; returns FTLM_ERR_UNSUPPORTED for cube_bits > 0 on other spins.
 */
ftlm_status ftlm_tune_shape(const ftlm_system* sys, int nvec, ftlm_dtype dtype, int cube_bits, int group_vectors,
                            int tile_cubes, int multipass);

const char* ftlm_last_error(void);
const char* ftlm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FTLM_H */
