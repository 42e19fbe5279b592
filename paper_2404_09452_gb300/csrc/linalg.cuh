// FP64 dense kernels of the DF-J/K build (linalg.cu).
#pragma once

#include <cuda_runtime.h>

namespace dfjk {

// C[b](m,n) = alpha sum_k A[b](m,k) B[b](n,k) + beta C[b](m,n), FP64, with
// element (m,k) of A at A + b sAb + m sAm + k sAk (same scheme for B, C).
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 1;
  const double *A = nullptr;
  long long sAm = 0, sAk = 0, sAb = 0;
  const double *B = nullptr;
  long long sBn = 0, sBk = 0, sBb = 0;
  double *C = nullptr;
  long long sCm = 0, sCn = 0, sCb = 0;
  double alpha = 1.0, beta = 0.0;
  int tile = 64;       // output tile edge: 64 (default) or 32 (4x more CTAs)
  int lower_only = 0;  // skip output tiles strictly above the diagonal
  int k_upto_n = 0;    // K range of an output tile limited to k < n_tile_end
                       // (B lower triangular in (n, k))
  int k_from_n = 0;    // K range starts at the tile's first n (B(n, k) = 0 for k < n)
  int k_upto_m = 0;    // K range ends at the tile's last m (A(m, k) = 0 for k > m)
  int k_from_m = 0;    // K range starts at the tile's first m (A(m, k) = 0 for k < m)
  int k_split = 0;     // >0: blockIdx.z selects K range [z k_split, ...) and C += z sCb
  // ragged diagonal-block batches: batch z has rag_n - (z rag_step + rag_off)
  // valid rows (and, with rag_clip_k, as many K); z with none returns
  int rag_n = 0, rag_step = 0, rag_off = 0, rag_clip_k = 0;
  // whitening epilogue: row m is column `m` of a T slab; writes
  // out[(mu nao + nu) ldo + n] and out[(nu nao + mu) ldo + n]
  const int *colmu = nullptr, *colnu = nullptr;
  int nao = 0;
  long long ldo = 0;
  double *out = nullptr;
};

void gemm_f64(const GemmArgs &g, cudaStream_t st);

// Diagonal block size of the blocked Cholesky and of the inverse's first level.
constexpr int CHOL_NB = 32;

// Cholesky of the lower triangle of A (n x n, n a multiple of CHOL_NB, lda),
// in place; Dinv (n / CHOL_NB blocks of CHOL_NB^2 doubles) receives the
// inverse of every diagonal block of L.  A non-positive pivot sets
// STATUS_NOT_PD in *status.
// With st2 and two events: look-ahead -- the next block column is updated on
// st (the critical chain of diagonal blocks and panels) while the rest of the
// trailing matrix is updated on st2; st waits for st2 before returning.
void cholesky_f64(double *A, int n, int lda, double *Dinv, int *status, double *work,
                  cudaStream_t st, cudaStream_t st2 = nullptr, cudaEvent_t ev_panel = nullptr,
                  cudaEvent_t ev_bulk = nullptr);
// Linv = L^-1 (lower triangular), n a multiple of CHOL_NB; uses Dinv from
// cholesky_f64 and `work` (n x n doubles).
void tri_inverse_f64(const double *L, int n, int ld, const double *Dinv, double *Linv,
                     double *work, cudaStream_t st);

// B storage: rows of ldb doubles (P contiguous), row(mu, nu) = mu nao + nu
// (both triangles stored, rowmap null) or rowmap[mu nao + nu] (the kept AO
// pairs only; -1 for a screened pair, whose B is zero).
//
// rho[P] = sum_{mu >= nu} w D[mu][nu] B[row ldb + P], w = 2 off the diagonal;
// partial sums in `work` (ceil(naux/256) x nchunk) then a fixed-order reduction.
void rho_gemv_f64(const double *B, long long ldb, int nao, int naux, const double *D,
                  double *rho, double *work, int nchunk, cudaStream_t st, const int *rowmap = nullptr);
// Both triangles of a row-mapped B: Bfull[(mu nao + nu) ldb + P] (nao^2 rows).
void unpack_rows_f64(const double *Bc, long long ldb, int nao, const int *rowmap, double *Bfull, cudaStream_t st);
// The row map of the kept columns: rowmap[mu nao + nu] = rowmap[nu nao + mu] =
// m for colmu[m] >= 0, -1 elsewhere (nao^2 ints).
void build_rowmap(const int *colmu, const int *colnu, long long ncol, int nao, int *rowmap, cudaStream_t st);
// rho[P] = sum_{mu,i} C[mu][i] X[mu][P][i]  (= sum_{mu nu} B[mu][nu][P] D[mu][nu]
// since X_P = B_P C and D = C C^T); per-mu partials in `part` (nao x np).
void rho_from_x_f64(const double *X, const double *C, int nao, int np, int nocc, double *rho,
                    double *part, cudaStream_t st);
// J[mu][nu] = J[nu][mu] = sum_P B[row(mu, nu) ldb + P] rho[P] for mu >= nu
// (0 for a screened pair).
void j_gemv_f64(const double *B, long long ldb, int nao, int naux, const double *rho, double *J,
                const int *rowmap, cudaStream_t st);
// out[mu][nu] = out[nu][mu] = sum_s part[s][mu][nu] (mu >= nu), summed in
// split order; add = 1 starts the sum from the current out[mu][nu].
void reduce_sym_f64(const double *part, int nsplit, int n, double *out, cudaStream_t st, int add = 0);
// K[mu][nu] = K[nu][mu] for nu > mu (the lower triangle is the result).
void mirror_lower_f64(double *K, int n, cudaStream_t st);
// e[0] = Tr(D J)/2, e[1] = Tr(D K)/2 (fixed-order two-level reduction).
void energies_f64(const double *D, const double *J, const double *K, int n, double *e,
                  double *work, cudaStream_t st);
// max_P sqrt(V[P][P]) over the first n diagonal entries.
void max_sqrt_diag(const double *V, int n, int ld, double *out, cudaStream_t st);
// keep[i] = q[i] * (*maxdiag) >= thresh
void screen_pairs(const double *q, int n, const double *maxdiag, double thresh, int *keep,
                  cudaStream_t st);
void fill_f64(double *p, long long n, double v, cudaStream_t st);
// out[i][j] = in[perm_r[i] * ldi + perm_c[j]] for an n_r x n_c gather (0 where
// perm_r[i] < 0).
void gather2d_f64(const double *in, long long ldi, const int *perm_r, const int *perm_c, int nr,
                  int nc, double *out, long long ldo, cudaStream_t st);
// B user-order copy: out[P][mu][nu] = Bint[row(mu, nu) ldb + perm[P]] (row as
// above).
void gather_B_f64(const double *Bint, long long ldb, int nao, const int *perm, int naux,
                  double *out, const int *rowmap, cudaStream_t st);

}  // namespace dfjk
