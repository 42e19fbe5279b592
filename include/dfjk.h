/*
 * dfjk.h -- C ABI of the GB300 density-fitted Coulomb/exchange (DF-J/K) build.
 *
 * The method (paper: Introduction, contribution 1; Sec. "Dataset and
 * Performance" on keeping intermediates resident in GPU memory; Sec.
 * "Improved Interfaces to External Libraries" on tensor-core contractions):
 * 3-centre integrals (P|mu nu) over contracted Cartesian Gaussians, whitened
 * with the Cholesky factor of the 2-centre metric (P|Q) = L L^T into
 * B = L^-1 (P|mu nu), then
 *     rho_P = sum_{mu nu} B[P][mu][nu] D[mu][nu],    J = B^T rho,
 *     X_P   = B_P C_occ,                             K = sum_P X_P X_P^T,
 *     E_J   = Tr(D J) / 2,  E_K = Tr(D K) / 2,       D = C_occ C_occ^T.
 * For one spin-orbital set D the restricted two-electron energy is
 * 4 E_J - 2 E_K (E_K here is the positive exchange energy of D).
 *
 * Conventions.  Units are bohr and hartree.  Shells are Cartesian with
 * 0 <= l <= 2; components are ordered x,y,z (l=1) and xx,xy,xz,yy,yz,zz (l=2);
 * AO order is shell order, then component.  Every Cartesian component is
 * normalised to unit self-overlap: primitive norm
 * (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!), and the contraction
 * is rescaled so <chi|chi> = 1.  Matrices are row-major FP64.
 *
 * Errors.  Every entry point returns an int status (DFJK_OK = 0).  A detail
 * message for the last failure on the calling thread is available from
 * dfjk_last_error().  No C++ exception crosses this boundary and device code
 * never traps: device-side failures (a non-positive Cholesky pivot, an
 * expired bounded wait) are written to a status word that the host reads.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  dfjk_build enqueues work and returns without synchronising;
 * outputs are valid once the stream reaches that point.  dfjk_setup
 * synchronises its stream twice (to size the screened pair list and to read
 * the Cholesky status) and returns with the handle's data resident.
 */
#ifndef DFJK_H
#define DFJK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DFJK_OK = 0,
  DFJK_ERR_ARG = 1,         /* invalid argument (null pointer, bad size)       */
  DFJK_ERR_UNSUPPORTED = 2, /* l > 2, nprim > 8, or a precision not built     */
  DFJK_ERR_NOT_PD = 3,      /* (P|Q) has a non-positive Cholesky pivot         */
  DFJK_ERR_OOM = 4,         /* device allocation failed                        */
  DFJK_ERR_BUDGET = 5,      /* resident data would exceed hbm_budget_bytes     */
  DFJK_ERR_TIMEOUT = 6,     /* a bounded device wait expired                   */
  DFJK_ERR_CUDA = 7,        /* a CUDA runtime call failed                      */
  DFJK_ERR_STATE = 8        /* handle used in the wrong state (e.g. evicted)   */
};

/* One contracted Cartesian shell (host memory, caller-owned; copied by
 * dfjk_setup).  coefs multiply *unnormalised* primitives; the library
 * applies the normalisation described above.                                */
typedef struct {
  int32_t atom;  /* index into coords                                       */
  int32_t l;     /* 0..2                                                    */
  int32_t nprim; /* 1..8                                                    */
  const double *exps;
  const double *coefs;
} dfjk_shell;

typedef struct {
  int32_t nshell;
  const dfjk_shell *shells;
} dfjk_basis;

/* Precision of a handle.  The paper moves its tensor contractions onto tensor
 * cores (Introduction, contribution 2: "up to twice the speed"; Sec.
 * "Improved Interfaces to External Libraries": cuTENSOR contractions on
 * tensor cores); DFJK_MIXED does the same for the three dense contractions
 * while keeping FP64-level results.                                          */
typedef enum {
  DFJK_FP64 = 0, /* every step in FP64 on the FP64 pipe (the plain path); B is
                    kept in both triangles, nao^2 naux_pad doubles            */
  DFJK_MIXED = 1 /* integrals (FP64; FP32 for the pairs below
                    fp32_pair_thresh), Cholesky and inverse, rho, J and the
                    energies in FP64.  B is kept in FP64 for the
                    Schwarz-kept AO pairs only, one row of naux_pad doubles
                    per kept column (a quarter of the mu >= nu pairs at 60
                    atoms, fewer for larger molecules).
                    The whitening, X = B C and K run on the tensor cores as
                    exact sliced products: each FP64 operand row is cut into 6
                    (8 for the whitening) 6-bit integer slices stored as BF16
                    (2 bytes per slice) under a power-of-two exponent per
                    1024-element block, products accumulate exactly in FP32
                    TMEM and are recombined in int64/FP64.  Each build slices
                    B again, chunk by chunk of aux rows P (work buffers of at
                    most DFJK_BUILD_WS_MB megabytes, default 8192, or 128 rows) */
} dfjk_precision;

typedef struct {
  int32_t precision;       /* dfjk_precision                                 */
  double schwarz_thresh;   /* drop shell pair ab if sqrt(max(ab|ab)) *
                              max_P sqrt((P|P)) < thresh; default 1e-12       */
  size_t hbm_budget_bytes; /* 0 = no limit; else setup fails with
                              DFJK_ERR_BUDGET if resident data would exceed it */
  int64_t timeout_iters;   /* iteration limit of bounded device waits        */
  int32_t energies_on_host;/* informational: dfjk_build detects whether its
                              E_J/E_K pointers are host memory (the call then
                              synchronises the stream) or device memory      */
  double fp32_pair_thresh; /* Schwarz-guided mixed precision of the 3-centre
                              integrals (the paper's future-work item in
                              "Limitations and Future Development"): kept
                              pairs whose bound sqrt(max(ab|ab)) *
                              max_P sqrt((P|P)) is below this value are
                              evaluated in FP32.  0 = every pair in FP64;
                              negative = the precision's default (0 for
                              DFJK_FP64, 1e-5 for DFJK_MIXED)                 */
  int32_t b_on_host;       /* 1: keep B in pinned host memory mapped into the
                              device address space (the kernels read and
                              write it in place over the host link; for
                              molecules whose B does not fit in device
                              memory: the paper's CPU-memory storage of the
                              intermediates of large systems, Sec. "Dataset
                              and Performance").  0 (default): B in device
                              memory                                        */
  const char *tune_table;  /* path of a tuning table (written by the
                              package's autotuner, tune.py): per range of
                              nao, rows per block of the slicing kernels, the
                              K GEMM's split-K range and the mixed build's
                              work-buffer cap; read during dfjk_setup (not
                              kept).  NULL: the DFJK_TUNE_TABLE environment
                              variable, else built-in defaults.  These only
                              change launch shapes: the slicing choices leave
                              results bitwise equal, the K range and the cap
                              regroup FP64 sums (differences ~1e-12)       */
} dfjk_options;

typedef struct dfjk_ctx *dfjk_handle;

/* Fills *opt with the defaults: DFJK_FP64, 1e-12, no budget, 1<<26, host
 * energies, fp32_pair_thresh -1 (the precision's default), B on the device,
 * no tuning table.                                                           */
void dfjk_default_options(dfjk_options *opt);

/* Setup: the first half of the paper's density-fitting scheme (Introduction,
 * contribution 1: the 3-centre integrals are computed first, everything after
 * them is tensor operations), with the intermediates of the molecule kept in
 * GPU memory (Sec. "Dataset and Performance").  Validates and normalises the
 * bases, builds the shell-pair list with Schwarz screening, the metric (P|Q),
 * its Cholesky factor and inverse, the 3-centre integrals and the whitened
 * tensor B, which stays resident on the current device until
 * dfjk_destroy/dfjk_evict.
 *   orb, aux : host shell lists (copied).  natom, coords: natom x 3 host doubles.
 *   opt      : may be NULL (defaults).  out: receives the handle.
 * Errors: DFJK_ERR_ARG, _UNSUPPORTED, _NOT_PD, _OOM, _BUDGET, _CUDA.           */
int dfjk_setup(const dfjk_basis *orb, const dfjk_basis *aux, int32_t natom,
               const double *coords, const dfjk_options *opt, void *stream,
               dfjk_handle *out);

/* Sizes of a handle: number of AOs, aux functions, screened shell pairs, and
 * device bytes it holds resident.  Any output pointer may be NULL.          */
int dfjk_query(dfjk_handle h, int32_t *nao, int32_t *naux, int32_t *npair_kept,
               size_t *device_bytes);

/* Precision split of the 3-centre integrals of a handle: the number of kept
 * shell pairs evaluated in FP32 and the bound threshold that selected them
 * (0 when every pair is FP64).  Either output pointer may be NULL.           */
int dfjk_query_precision(dfjk_handle h, int32_t *npair_fp32, double *fp32_thresh);

/* Work of a handle's 3-centre integrals: the kept primitive pairs of each
 * orbital shell-pair class (ss, ps, pp, ds, dp, dd), evaluated in FP64
 * (prim_pairs_fp64[6]) and in FP32 (prim_pairs_fp32[6]).  Each meets every
 * aux primitive once (one primitive triple).  Either pointer may be NULL.   */
int dfjk_query_pair_classes(dfjk_handle h, int64_t *prim_pairs_fp64, int64_t *prim_pairs_fp32);

/* The launch-shape choices a handle took from its tuning table, vals[4] =
 * {slicing rows per block, B slicing rows per block, K GEMM split-K
 * range in MB, build work-buffer cap in MB}; 0 = the built-in default.       */
int dfjk_query_tuning(dfjk_handle h, int32_t *vals);

/* Layout of a handle's setup: the number of 3-centre column slabs (T is
 * built and whitened slab by slab, at most 4 GiB each, 2 GiB in the mixed
 * path) and whether B holds rows for the Schwarz-kept AO pairs only (1 for
 * every DFJK_MIXED handle; 0 for DFJK_FP64, whose B has both triangles of
 * every pair).  Either output pointer may be NULL.                           */
int dfjk_query_setup(dfjk_handle h, int32_t *nslab, int32_t *lean);

/* Aux-row chunking of the DFJK_MIXED build (the build slices B, forms X and
 * adds its K contribution chunk by chunk of rows P, one X and one K GEMM
 * launch per chunk): rows per chunk and the number of chunks, both 0 before
 * the handle's first build and for DFJK_FP64.  Either pointer may be NULL.   */
int dfjk_query_build(dfjk_handle h, int32_t *chunk_rows, int32_t *nchunk);

/* Device bytes a molecule with nao AOs and naux aux functions takes at the
 * given precision, before any setup (no device work): `resident` = what a
 * handle holds between builds (B and the metric, its Cholesky factor and
 * inverse; for DFJK_MIXED an upper bound that counts every mu >= nu pair as
 * kept, dfjk_query gives a set-up handle's actual bytes), `build_ws` = the
 * work buffers a build at nocc occupied orbitals
 * adds (kept by the handle for its next builds), `setup_ws` = the transient
 * peak of the setup beyond the resident data (released when it returns).
 * Used to admit molecules under a memory budget (batching, serving).
 * Any output pointer may be NULL.  Errors: DFJK_ERR_ARG.                     */
int dfjk_estimate_bytes(int32_t nao, int32_t naux, int32_t nocc, int32_t precision, size_t *resident,
                        size_t *build_ws, size_t *setup_ws);

/* Build: the tensor-operation half of the paper's density-fitting scheme
 * (Introduction, contribution 1) for nset occupied-orbital sets:
 * X_P = B_P C, K = sum_P X_P X_P^T, rho = B vec(D), J = B^T rho, energies.
 *   C_occ : device, nset x nao x nocc, row-major FP64 (caller-owned).
 *   J, K  : device, nset x nao x nao FP64, written in full (symmetric).
 *   E_J, E_K : nset doubles each, both host or both device memory (detected;
 *              host memory makes the call synchronise the stream).
 * Work buffers are owned by the handle and reused across calls; calls on one
 * handle must therefore be ordered on a stream.                              */
int dfjk_build(dfjk_handle h, int32_t nset, int32_t nocc, const double *C_occ,
               double *J, double *K, double *E_J, double *E_K, void *stream);

/* J and K from densities instead of orbitals: J = B^T (B vec D) and
 * K = sum_P B_P D B_P, for any symmetric D (not necessarily C C^T), on the
 * FP64 pipe whatever the handle's precision (two GEMMs of nao^3 naux each, so
 * much slower than dfjk_build).
 *   D    : device, nset x nao x nao FP64, symmetric.
 *   J, K : device, nset x nao x nao FP64.
 *   E_J, E_K : nset doubles each, Tr(D J)/2 and Tr(D K)/2, host or device.
 * Uses a work buffer of nao^2 naux_pad doubles for the duration of the call,
 * and for a DFJK_MIXED handle (B of the kept pairs only) a second one holding
 * B in both triangles of every pair; synchronises the stream before
 * returning.  Errors:
 * DFJK_ERR_ARG, _OOM, _CUDA.                            */
int dfjk_build_density(dfjk_handle h, int32_t nset, const double *D, double *J, double *K,
                       double *E_J, double *E_K, void *stream);

/* Nuclear gradient of the density-fitted Coulomb energy at fixed density,
 * E_J = u^T V^-1 u / 2 with u_P = sum_{mu nu} (P|mu nu) D_mu nu (the E_J of
 * dfjk_build / dfjk_build_density): the Coulomb part of the analytic
 * density-fitted SCF gradient, one of the three modules the paper benchmarks
 * (SCF, gradient, Hessian), computed as
 *   dE_J/dR = sum_P d_P du_P/dR - d^T (dV/dR) d / 2,   d = V^-1 u = L^-T rho,
 * with derivative 3-centre and 2-centre integrals over the kept shell pairs:
 * FP64, except that a DFJK_MIXED handle evaluates the pairs whose integrals
 * its build evaluates in FP32 (Schwarz bound below fp32_pair_thresh) in FP32
 * too, accumulated in FP64.  The AO density is
 * held fixed (no orbital response or overlap-derivative term: those belong to
 * the full SCF gradient, not to the Coulomb build).
 *   D    : device nao x nao FP64, symmetric (e.g. C C^T).
 *   grad : device natom x 3 FP64, overwritten; atoms in the order of the
 *          coordinates given to dfjk_setup.
 * Allocates small work buffers and synchronises the stream before returning.
 * Errors: DFJK_ERR_ARG, _OOM, _CUDA.                                          */
int dfjk_coulomb_gradient(dfjk_handle h, const double *D, double *grad, void *stream);

/* Nuclear gradient of c_j E_J + c_k E_K at fixed D = C C^T, E_J and E_K as
 * returned by dfjk_build (E_K = Tr(D K)/2, K = sum_P B_P D B_P).  Both are
 * E = sum_PQ (V^-1)_PQ M_PQ / 2 with M_PQ = u_P u_Q or Tr(D T_P D T_Q), so
 *   dE/dR = sum_P Tr(G_P dT_P/dR) - Tr(W dV/dR) / 2,
 * G_P = d_P D (J) or C Z_P C^T (K), W = d d^T (J) or Z Z^T (K), with
 * Z_P = sum_Q (L^-1)_QP C^T B_Q C (nocc x nocc per aux function).  The
 * derivative integrals are FP64 when c_k != 0 (with c_k = 0 the precision
 * split of dfjk_coulomb_gradient applies); the K part's contractions (X = B C, C^T X,
 * Z, Z Z^T, C Z_P C^T) run on the FP64 pipe for a DFJK_FP64 handle and as
 * exact sliced tensor-core products (as in the build) for a DFJK_MIXED one.
 * The K part holds Z, W (naux_pad^2) and G (naux_pad x nao^2 doubles, the
 * size of B), plus their sliced forms, for the duration of the call.
 *   C_occ : device nao x nocc FP64 row-major, 1 <= nocc <= nao.
 *   c_j, c_k : finite weights of E_J and E_K (c_k = 0 skips the K part).
 *   grad : device natom x 3 FP64, overwritten.
 * Synchronises the stream.  Errors: DFJK_ERR_ARG, _OOM, _CUDA.               */
int dfjk_jk_gradient(dfjk_handle h, int32_t nocc, const double *C_occ, double c_j, double c_k, double *grad,
                     void *stream);

/* Spin-unrestricted build: two occupied sets, alpha and beta, with their own
 * counts (the "unrestricted" row of the paper's functionality table, Sec.
 * "Accelerated Functionalities", marked optimised for SCF, gradient and
 * Hessian).  D_a = C_a C_a^T, D_b = C_b C_b^T.
 *   C_a : device nao x nocc_a, C_b : device nao x nocc_b (row-major FP64);
 *         1 <= nocc_a, 0 <= nocc_b <= nocc_a (nocc_b = 0: C_b may be NULL).
 *   J   : device nao x nao, Coulomb matrix of the total density D_a + D_b.
 *   K_a, K_b : device nao x nao, exchange matrices of each spin (K_b = 0 when
 *         nocc_b = 0).
 *   E   : 3 doubles, host or device (detected): E[0] = Tr((D_a + D_b) J)/2,
 *         E[1] = Tr(D_a K_a)/2, E[2] = Tr(D_b K_b)/2; the two-electron energy
 *         of the determinant is E[0] - E[1] - E[2].
 * Same buffers, ordering and errors as dfjk_build.                          */
int dfjk_build_uks(dfjk_handle h, int32_t nocc_a, const double *C_a, int32_t nocc_b,
                   const double *C_b, double *J, double *K_a, double *K_b, double *E,
                   void *stream);

/* dfjk_build for nmol resident handles at once (batching many molecules of
 * uneven size on one GPU; the paper runs one molecule per job and has no
 * counterpart): the builds
 * are spread over `nstreams` internal streams forked from and joined back to
 * `stream`, so small molecules run concurrently.  Handle i uses nocc[i],
 * C_occ[i] (device nao_i x nocc_i), J[i], K[i] (device nao_i x nao_i), and
 * writes E_J[i], E_K[i] (device arrays of nmol doubles).  No host
 * synchronisation: once each handle has been built at its nocc before (so
 * its work buffers exist), the call can be captured in a CUDA graph.  Each
 * handle may appear once per call.  Errors: DFJK_ERR_ARG, _STATE (evicted).  */
int dfjk_build_batch(int32_t nmol, const dfjk_handle *hs, const int32_t *nocc,
                     const double *const *C_occ, double *const *J, double *const *K,
                     double *E_J, double *E_K, int32_t nstreams, void *stream);

/* Overlap matrix S (device, nao x nao), computed by a device kernel; used to
 * orthonormalise occupied orbitals.                                           */
int dfjk_overlap(dfjk_handle h, double *S, void *stream);

/* Overlap matrix of a basis without a handle (no setup): S device nao x nao.
 * Used to prepare orthonormal occupied orbitals for many molecules.         */
int dfjk_overlap_matrix(const dfjk_basis *orb, int32_t natom, const double *coords, double *S,
                        void *stream);

/* Frees B and the work buffers but keeps the host copy of the inputs, so a
 * later dfjk_build recomputes the setup first (resident-set eviction: the
 * paper keeps the intermediates of small molecules in GPU memory and those
 * of large ones elsewhere, Sec. "Dataset and Performance"; a server that
 * holds many molecules under a memory budget evicts and recomputes).        */
int dfjk_evict(dfjk_handle h);

/* Releases everything the handle owns.  NULL is accepted.                    */
int dfjk_destroy(dfjk_handle h);

const char *dfjk_status_string(int code);
const char *dfjk_last_error(void);

/* Measured fused multiply-add throughput of the current GPU in TFLOP/s
 * (2 flop per FMA), bits = 64 (FP64 pipe) or 32 (FP32 pipe): independent FMA
 * chains on every SM, the best of four occupancy / chain-count shapes, each
 * timed for about 40 ms after three calibration launches.  The
 * roofline of the integral kernels, which are bound by these pipes.
 * Synchronises `stream`.  Errors: DFJK_ERR_ARG, _CUDA.                     */
int dfjk_fma_rate(int32_t bits, double *tflops, void *stream);

/* Number of kernels this library has launched in this process.             */
uint64_t dfjk_launch_count(void);

/* Phase timing (process-wide).  dfjk_set_timing(1) makes every later call
 * record a CUDA event pair around each phase, on the stream the phase is
 * launched on; dfjk_phase_times waits for those events, writes the
 * accumulated milliseconds of phases 0..n-1 to ms[] and clears them.
 * Phases: 0 shell pairs + Schwarz + metric, 1 Cholesky + inverse,
 * 2 3-centre integrals, 3 whitening, 4 X = B C (with the per-build slicing
 * of B), 5 K = sum X X^T, 6 D, rho and J, 7 energies; in
 * DFJK_MIXED also the tensor-core GEMM launches alone: 8 whitening, 9 X = B C,
 * 10 K (each also counted inside phases 3, 4, 5); 11 the 3-centre integrals
 * of the shell pairs evaluated in FP32 (phase 2 then holds the FP64 ones);
 * 12 the whole setup and 13 the whole build, each from its first to its last
 * operation on the call's stream (the time between them is host work).      */
#define DFJK_NPHASE 14
int dfjk_set_timing(int32_t enable);

/* Frees the device blocks the library keeps cached for reuse after handles
 * release them (the cache holds at most DFJK_CACHE_BYTES per device,
 * environment variable, default 96 GiB).                                     */
int dfjk_trim_cache(void);
int dfjk_phase_times(double *ms, int32_t n);

/* ---- diagnostic accessors (tests and parity checks) ---------------------- */

/* F_m(T) for m = 0..mmax at n points: T device [n], F device [n][mmax+1].
 * mmax <= 8.                                                                 */
int dfjk_boys(int32_t mmax, int32_t n, const double *T, double *F, void *stream);

/* Copies of resident intermediates, in user AO / aux order, device FP64:
 *   V, L : naux x naux (L lower triangular, zero above the diagonal)
 *   B    : naux x nao x nao (whitened tensor, expanded to FP64)
 *   keep : nshell_orb x nshell_orb int32, 1 where the shell pair survived
 *          Schwarz screening (symmetric)                                     */
int dfjk_get_metric(dfjk_handle h, double *V, void *stream);
int dfjk_get_cholesky(dfjk_handle h, double *L, void *stream);
int dfjk_get_B(dfjk_handle h, double *B, void *stream);
int dfjk_get_pair_mask(dfjk_handle h, int32_t *keep, void *stream);

/* Columns of B without expanding all of it (for checks at sizes where the
 * full naux x nao x nao copy would not fit): out[c][P] = B[P][mu[c]][nu[c]],
 * c < ncol, P < naux.  mu, nu: host int32 arrays; out: device FP64
 * ncol x naux.  Synchronises the stream.                                     */
int dfjk_get_B_columns(dfjk_handle h, int32_t ncol, const int32_t *mu, const int32_t *nu, double *out,
                       void *stream);

/* Raw 3-centre integrals T[P][mu][nu] (before whitening), device FP64
 * naux x nao x nao; recomputed on demand.                                    */
int dfjk_get_three_center(dfjk_handle h, double *T, void *stream);

/* The exact sliced-product tensor-core GEMM used by DFJK_MIXED, on its own:
 * C[z][m][n] = sum_k A[z][m][k] B[n][k] with A (batch x M x K), B (N x K),
 * C (batch x M x N) device FP64 row-major; S = 6 or 8 slices of 6 bits per
 * operand row and 1024-wide K block.  Allocates its slice buffers, synchronises
 * `stream`.  *status (device int, may be NULL) receives STATUS bits.         */
int dfjk_debug_sliced_gemm(int32_t batch, int32_t M, int32_t N, int32_t K, int32_t S,
                           const double *A, const double *B, double *C, int32_t *status,
                           void *stream);

/* ---- allocation-free variant ------------------------------------------------ */

/* E[0] = sum_ij D_ij J_ij / 2 and E[1] = sum_ij D_ij K_ij / 2 for
 * caller-owned device matrices D, J, K (n x n FP64, row-major) into E
 * (device, 2 doubles), allocating nothing.  For the symmetric J and K that
 * dfjk_build writes these are Tr(D J)/2 and Tr(D K)/2; for a non-symmetric
 * J or K they are Tr(D J^T)/2 and Tr(D K^T)/2.  For callers that must not call cudaMalloc: an application whose
 * memory pool already owns the device memory, or code that cannot take the
 * device-wide synchronisation of cudaMalloc/cudaFree.  The paper has no
 * counterpart.
 *   Scratch: a 256 KB static device array inside this library (every GPU that
 *   loads the library holds it until exit).  The first call on each device
 *   looks up its address (cudaGetSymbolAddress) with that device current;
 *   make that first call before any stream capture.  All calls share the
 *   array and each call writes every slot it later reads; calls that overlap
 *   on the GPU race on it.
 *   Limit: n <= 8192; larger n returns DFJK_ERR_ARG without launching.
 *   Enqueued on `stream`; E is valid once the stream reaches this point.     */
int dfjk_energies_noalloc(int32_t n, const double *D, const double *J, const double *K,
                          double *E, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DFJK_H */
