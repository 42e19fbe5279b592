// FP64 dense kernels of the DF-J/K build: a generic strided GEMM (64x64x16
// tiles, 4x4 outputs per thread), blocked Cholesky and triangular inverse of
// the metric, the two streaming GEMVs of J (rho = B vec(D), J = B^T rho) and
// deterministic reductions.
//
// Paper: Introduction, contribution 1 (after the 3-centre integrals, density
// fitting is tensor operations) and the accuracy passage of the PySCF
// compatibility section (the fitting solve).  On this GPU FP64 runs at about
// 1.2 TFLOP/s, 1/62 of FP32, so these SIMT kernels are bound by the FP64 pipe
// at any reasonable tiling; they are the plain-FP64 reference path.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "linalg.cuh"

namespace dfjk {

constexpr int GBK = 16;

// TILE x TILE output tile per 256-thread CTA, (TILE/16)^2 outputs per thread;
// TILE = 32 gives four times more CTAs for the small, latency-bound GEMMs of
// the Cholesky factorisation and the triangular inverse.
template <int TILE, bool A_KC, bool B_KC, bool SCATTER>
__global__ void __launch_bounds__(256) gemm_f64_kernel(GemmArgs g) {
  constexpr int GBM = TILE, GBN = TILE, TT = TILE / 16;
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  if (g.lower_only && n0 > m0 + GBM - 1) return;
  const int z = blockIdx.z;
  const double *A = g.A, *B = g.B;
  double *C = g.C;
  long long kbeg = 0, kend = g.K;
  if (g.k_split > 0) {
    kbeg = (long long)z * g.k_split;
    kend = min((long long)g.K, kbeg + g.k_split);
    C += z * g.sCb;
  } else {
    A += z * g.sAb;
    B += z * g.sBb;
    C += z * g.sCb;
  }
  if (g.k_upto_n) kend = min(kend, (long long)(n0 + GBN));
  if (g.k_upto_m) kend = min(kend, (long long)(m0 + GBM));
  if (g.k_from_n) kbeg = max(kbeg, (long long)n0);
  if (g.k_from_m) kbeg = max(kbeg, (long long)m0);
  int Mz = g.M;
  if (g.rag_step > 0) {
    const int valid = g.rag_n - (z * g.rag_step + g.rag_off);
    if (valid <= 0 || m0 >= valid) return;
    Mz = min(Mz, valid);
    if (g.rag_clip_k) kend = min(kend, (long long)valid);
  }
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) acc[i][j] = 0.0;

  for (long long k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int i = 0; i < TT; ++i) {
      const int e = tid + i * 256;
      const int mm = A_KC ? (e >> 4) : (e % GBM);
      const int kk = A_KC ? (e & 15) : (e / GBM);
      const long long gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < Mz && gk < kend) ? A[gm * g.sAm + gk * g.sAk] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < TT; ++i) {
      const int e = tid + i * 256;
      const int nn = B_KC ? (e >> 4) : (e % GBN);
      const int kk = B_KC ? (e & 15) : (e / GBN);
      const long long gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < g.N && gk < kend) ? B[gn * g.sBn + gk * g.sBk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[TT], b[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) a[i] = As[kk][ty * TT + i];
#pragma unroll
      for (int j = 0; j < TT; ++j) b[j] = Bs[kk][tx * TT + j];
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TT; ++i) {
    const int m = m0 + ty * TT + i;
    if (m >= Mz) continue;
    if (SCATTER) {
      const int mu = g.colmu[m], nu = g.colnu[m];
      if (mu < 0) continue;
      double *o1 = g.out + ((long long)mu * g.nao + nu) * g.ldo;
      double *o2 = g.out + ((long long)nu * g.nao + mu) * g.ldo;
#pragma unroll
      for (int j = 0; j < TT; ++j) {
        const int n = n0 + tx * TT + j;
        if (n < g.N) {
          o1[n] = acc[i][j];
          if (mu != nu) o2[n] = acc[i][j];
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < TT; ++j) {
        const int n = n0 + tx * TT + j;
        if (n >= g.N) continue;
        double *c = C + m * g.sCm + n * g.sCn;
        *c = (g.beta != 0.0) ? fma(g.alpha, acc[i][j], g.beta * *c) : g.alpha * acc[i][j];
      }
    }
  }
}

template <int TILE>
static void gemm_f64_launch(const GemmArgs &g, cudaStream_t st) {
  const int nz = g.k_split > 0 ? ceil_div(g.K, g.k_split) : g.batch;
  if (nz <= 0) return;
  dim3 grid(ceil_div(g.N, TILE), ceil_div(g.M, TILE), nz);
  if (grid.y > 65535 || grid.z > 65535) throw Error{DFJK_ERR_ARG, "gemm grid too large"};
  const bool akc = g.sAk == 1, bkc = g.sBk == 1, sc = g.out != nullptr;
  if (sc) {
    if (akc && bkc) gemm_f64_kernel<TILE, true, true, true><<<grid, 256, 0, st>>>(g);
    else throw Error{DFJK_ERR_ARG, "scatter gemm needs K-contiguous operands"};
  } else if (akc && bkc) {
    gemm_f64_kernel<TILE, true, true, false><<<grid, 256, 0, st>>>(g);
  } else if (akc && !bkc) {
    gemm_f64_kernel<TILE, true, false, false><<<grid, 256, 0, st>>>(g);
  } else if (!akc && bkc) {
    gemm_f64_kernel<TILE, false, true, false><<<grid, 256, 0, st>>>(g);
  } else {
    gemm_f64_kernel<TILE, false, false, false><<<grid, 256, 0, st>>>(g);
  }
  DFJK_LAUNCHED();
}

void gemm_f64(const GemmArgs &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return;
  if (g.tile == 32) gemm_f64_launch<32>(g, st);
  else gemm_f64_launch<64>(g, st);
}

// ---- Cholesky -------------------------------------------------------------------

// Factors the NB x NB lower block at A in place (upper part zeroed) and writes
// its inverse (lower triangular) to Dinv.  A non-positive or non-finite pivot
// sets STATUS_NOT_PD and continues with pivot 1 so no NaN spreads.  The block
// runs on one SM, whose FP64 rate is 1/152 of the GPU's, so NB is kept small
// (32): the panel and trailing updates, spread over all SMs, do the bulk.
// Dynamic shared memory: two NB x (NB + 1) FP64 arrays.
template <int NB>
__global__ void __launch_bounds__(256) potrf_diag_kernel(double *A, int lda, double *Dinv,
                                                         int *status) {
  extern __shared__ double psm[];
  double(*a)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(psm);
  double(*x)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(psm + NB * (NB + 1));
  __shared__ double rdiag[NB];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < NB * NB; e += 256) {
    const int i = e / NB, j = e % NB;
    a[i][j] = (j <= i) ? A[(long long)i * lda + j] : 0.0;
    x[i][j] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    if (tid == 0) {
      double d = a[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(status, STATUS_NOT_PD);
        d = 1.0;
      }
      const double l = sqrt(d);
      a[j][j] = l;
      rdiag[j] = 1.0 / l;
    }
    __syncthreads();
    const double r = rdiag[j];
    if (tid > j && tid < NB) a[tid][j] *= r;
    __syncthreads();
    for (int i = j + 1 + ty; i < NB; i += 16) {
      const double lij = a[i][j];
      for (int c = j + 1 + tx; c <= i; c += 16) a[i][c] = fma(-lij, a[c][j], a[i][c]);
    }
    __syncthreads();
  }
  // X = L^-1 row by row: x[k][c] = -(sum_{c<=j<k} l[k][j] x[j][c]) / l[k][k];
  // four lanes share each dot product.
  const int c = tid >> 2, part = tid & 3;
  for (int k = 0; k < NB; ++k) {
    double sum = 0.0;
    if (c < k)
      for (int j = c + part; j < k; j += 4) sum = fma(a[k][j], x[j][c], sum);
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    if (part == 0 && c <= k) x[k][c] = (c == k) ? rdiag[k] : -sum * rdiag[k];
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += 256) {
    const int i = e / NB, j = e % NB;
    A[(long long)i * lda + j] = a[i][j];
    Dinv[e] = x[i][j];
  }
}

void cholesky_f64(double *A, int n, int lda, double *Dinv, int *status, double *work,
                  cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_panel, cudaEvent_t ev_bulk) {
  (void)work;
  constexpr int NB = CHOL_NB;
  constexpr int SMEM = 2 * NB * (NB + 1) * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    DFJK_CUDA_CHECK(cudaFuncSetAttribute(potrf_diag_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    attr = true;
  }
  const bool ahead = st2 && ev_panel && ev_bulk;
  const int nb = n / NB;
  bool bulk_pending = false;
  for (int k = 0; k < nb; ++k) {
    double *Akk = A + (long long)k * NB * lda + k * NB;
    potrf_diag_kernel<NB><<<1, 256, SMEM, st>>>(Akk, lda, Dinv + (long long)k * NB * NB, status);
    DFJK_LAUNCHED();
    const int rows = n - (k + 1) * NB;
    if (rows <= 0) continue;
    double *panel = A + (long long)(k + 1) * NB * lda + k * NB;
    GemmArgs p;  // L_ik = A_ik Dinv_k^T, in place (one tile owns complete rows)
    p.M = rows; p.N = NB; p.K = NB;
    p.A = panel; p.sAm = lda; p.sAk = 1;
    p.B = Dinv + (long long)k * NB * NB; p.sBn = NB; p.sBk = 1;
    p.C = panel; p.sCm = lda; p.sCn = 1;
    // tile = the whole panel width: the update is in place, so one CTA must
    // own complete rows (with narrower tiles two CTAs would share them)
    p.tile = NB;
    gemm_f64(p, st);
    if (!ahead) {
      GemmArgs t;  // A_ij -= L_ik L_jk^T on the trailing lower triangle
      t.M = rows; t.N = rows; t.K = NB;
      t.A = panel; t.sAm = lda; t.sAk = 1;
      t.B = panel; t.sBn = lda; t.sBk = 1;
      t.C = A + (long long)(k + 1) * NB * (lda + 1); t.sCm = lda; t.sCn = 1;
      t.alpha = -1.0; t.beta = 1.0; t.lower_only = 1;
      t.tile = 32;
      gemm_f64(t, st);
      continue;
    }
    // look-ahead: the next block column (k + 1) is updated on the critical
    // stream, so the next diagonal block can start, while the rest of the
    // trailing matrix (block columns >= k + 2) is updated on the second
    // stream; block column k + 1 also receives the second stream's earlier
    // updates, which must have landed first
    DFJK_CUDA_CHECK(cudaEventRecord(ev_panel, st));
    if (bulk_pending) DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, ev_bulk, 0));
    GemmArgs c;  // A_{i,k+1} -= L_ik L_{k+1,k}^T for block rows i >= k + 1
    c.M = rows; c.N = NB; c.K = NB;
    c.A = panel; c.sAm = lda; c.sAk = 1;
    c.B = panel; c.sBn = lda; c.sBk = 1;
    c.C = A + (long long)(k + 1) * NB * (lda + 1); c.sCm = lda; c.sCn = 1;
    c.alpha = -1.0; c.beta = 1.0;
    c.tile = 32;
    gemm_f64(c, st);
    const int rest = rows - NB;
    if (rest > 0) {
      DFJK_CUDA_CHECK(cudaStreamWaitEvent(st2, ev_panel, 0));
      GemmArgs t;  // A_ij -= L_ik L_jk^T for block rows and columns >= k + 2
      t.M = rest; t.N = rest; t.K = NB;
      t.A = panel + (long long)NB * lda; t.sAm = lda; t.sAk = 1;
      t.B = panel + (long long)NB * lda; t.sBn = lda; t.sBk = 1;
      t.C = A + (long long)(k + 2) * NB * (lda + 1); t.sCm = lda; t.sCn = 1;
      t.alpha = -1.0; t.beta = 1.0; t.lower_only = 1;
      t.tile = 32;
      gemm_f64(t, st2);
      DFJK_CUDA_CHECK(cudaEventRecord(ev_bulk, st2));
      bulk_pending = true;
    }
  }
  if (bulk_pending) DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, ev_bulk, 0));
}

__global__ void place_diag_blocks(double *Linv, int ld, const double *Dinv, int nb) {
  constexpr int NB = CHOL_NB;
  const int b = blockIdx.x;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    Linv[((long long)b * NB + i) * ld + b * NB + j] = Dinv[(long long)b * NB * NB + e];
  }
}

// L^-1 bottom-up: at level s the already inverted diagonal blocks of size s
// are merged in pairs (rows [j 2s, j 2s + s) and [j 2s + s, min(n, j 2s + 2s)));
// the lower-left block of the merged inverse is -Linv22 (L21 Linv11).  All
// pairs of a level run in one batched launch; the ragged last pair is clipped
// in the kernel.
void tri_inverse_f64(const double *L, int n, int ld, const double *Dinv, double *Linv,
                     double *work, cudaStream_t st) {
  DFJK_CUDA_CHECK(cudaMemsetAsync(Linv, 0, sizeof(double) * (size_t)n * ld, st));
  const int nb = n / CHOL_NB;
  place_diag_blocks<<<nb, 256, 0, st>>>(Linv, ld, Dinv, nb);
  DFJK_LAUNCHED();
  for (int s = CHOL_NB; s < n; s *= 2) {
    const int pairs = (n + 2 * s - 1) / (2 * s);
    const long long dstep = 2LL * s * (ld + 1);
    GemmArgs a;  // work_j = L21_j Linv11_j   (rows clipped to the valid part of block 2)
    a.M = s; a.N = s; a.K = s; a.batch = pairs;
    a.A = L + (long long)s * ld; a.sAm = ld; a.sAk = 1; a.sAb = dstep;
    a.B = Linv; a.sBn = 1; a.sBk = ld; a.sBb = dstep;
    a.C = work; a.sCm = s; a.sCn = 1; a.sCb = (long long)s * s;
    a.rag_n = n; a.rag_step = 2 * s; a.rag_off = s;
    a.k_from_n = 1;  // Linv11 lower triangular: B(n, k) = Linv11[k][n] = 0 for k < n
    a.tile = 32;
    gemm_f64(a, st);
    GemmArgs b;  // Linv21_j = -Linv22_j work_j
    b.M = s; b.N = s; b.K = s; b.batch = pairs;
    b.A = Linv + (long long)s * ld + s; b.sAm = ld; b.sAk = 1; b.sAb = dstep;
    b.B = work; b.sBn = 1; b.sBk = s; b.sBb = (long long)s * s;
    b.C = Linv + (long long)s * ld; b.sCm = ld; b.sCn = 1; b.sCb = dstep;
    b.alpha = -1.0;
    b.rag_n = n; b.rag_step = 2 * s; b.rag_off = s; b.rag_clip_k = 1;
    b.k_upto_m = 1;  // Linv22 lower triangular: A(m, k) = 0 for k > m
    b.tile = 32;
    gemm_f64(b, st);
  }
}

// ---- J: rho = B vec(D), J = B^T rho ------------------------------------------------

__device__ __forceinline__ void tri_row(long long r, int &mu, int &nu) {
  int m = (int)((sqrt(8.0 * (double)r + 1.0) - 1.0) * 0.5);
  while ((long long)m * (m + 1) / 2 > r) --m;
  while ((long long)(m + 1) * (m + 2) / 2 <= r) ++m;
  mu = m;
  nu = (int)(r - (long long)m * (m + 1) / 2);
}

__global__ void __launch_bounds__(256) rho_partial_kernel(const double *__restrict__ B,
                                                          long long ldb, int nao, int naux,
                                                          const double *__restrict__ D,
                                                          double *__restrict__ work, int ldw,
                                                          long long rows_per, const int *__restrict__ rowmap) {
  const int P = blockIdx.x * 256 + threadIdx.x;
  const long long nrows = (long long)nao * (nao + 1) / 2;
  const long long r0 = (long long)blockIdx.y * rows_per;
  const long long r1 = min(nrows, r0 + rows_per);
  double acc = 0.0;
  if (r0 < r1) {
    int mu, nu;
    tri_row(r0, mu, nu);
    for (long long r = r0; r < r1; ++r) {
      const double w = D[(long long)mu * nao + nu] * (mu == nu ? 1.0 : 2.0);
      const long long row = rowmap ? rowmap[(long long)mu * nao + nu] : (long long)mu * nao + nu;
      if (P < naux && row >= 0) acc = fma(w, B[row * ldb + P], acc);
      if (++nu > mu) {
        ++mu;
        nu = 0;
      }
    }
  }
  if (P < ldw) work[(long long)blockIdx.y * ldw + P] = acc;
}

__global__ void column_sum_kernel(const double *__restrict__ work, int ldw, int nrow, int n,
                                  double *__restrict__ out) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= n) return;
  double s = 0.0;
  for (int r = 0; r < nrow; ++r) s += work[(long long)r * ldw + P];
  out[P] = s;
}

void rho_gemv_f64(const double *B, long long ldb, int nao, int naux, const double *D,
                  double *rho, double *work, int nchunk, cudaStream_t st, const int *rowmap) {
  const long long nrows = (long long)nao * (nao + 1) / 2;
  const long long rows_per = (nrows + nchunk - 1) / nchunk;
  const int gx = ceil_div(naux, 256), ldw = gx * 256;
  rho_partial_kernel<<<dim3(gx, nchunk), 256, 0, st>>>(B, ldb, nao, naux, D, work, ldw, rows_per, rowmap);
  DFJK_LAUNCHED();
  column_sum_kernel<<<ceil_div(naux, 256), 256, 0, st>>>(work, ldw, nchunk, naux, rho);
  DFJK_LAUNCHED();
}

// part[mu][P] = sum_i C[mu][i] X[mu][P][i]: one warp per (mu, P), lanes along i.
__global__ void __launch_bounds__(256) rho_from_x_kernel(const double *__restrict__ X,
                                                         const double *__restrict__ C, int nao, int np,
                                                         int nocc, double *__restrict__ part) {
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nao * np) return;
  const int mu = (int)(w / np);
  const double *x = X + w * nocc;
  const double *c = C + (long long)mu * nocc;
  double s = 0.0;
  for (int i = lane; i < nocc; i += 32) s = fma(__ldg(c + i), x[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[w] = s;
}

void rho_from_x_f64(const double *X, const double *C, int nao, int np, int nocc, double *rho,
                    double *part, cudaStream_t st) {
  const long long n = (long long)nao * np;
  rho_from_x_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(X, C, nao, np, nocc, part);
  DFJK_LAUNCHED();
  column_sum_kernel<<<ceil_div(np, 256), 256, 0, st>>>(part, np, nao, np, rho);
  DFJK_LAUNCHED();
}

__global__ void __launch_bounds__(256) j_gemv_kernel(const double *__restrict__ B, long long ldb,
                                                     int nao, int naux,
                                                     const double *__restrict__ rho,
                                                     double *__restrict__ J, const int *__restrict__ rowmap) {
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const long long nrows = (long long)nao * (nao + 1) / 2;
  if (r >= nrows) return;
  int mu, nu;
  tri_row(r, mu, nu);
  const long long br = rowmap ? rowmap[(long long)mu * nao + nu] : (long long)mu * nao + nu;
  const double *row = B + (br < 0 ? 0 : br) * ldb;
  double s = 0.0;
  if (br < 0) {  // a screened pair: no row stored, J is 0
  } else if ((naux & 1) == 0 && (ldb & 1) == 0) {  // 16-byte loads, two partial sums, 4 loads in flight
    const double2 *row2 = reinterpret_cast<const double2 *>(row);
    const double2 *rho2 = reinterpret_cast<const double2 *>(rho);
    double s1 = 0.0;
#pragma unroll 4
    for (int q = lane; q < naux / 2; q += 32) {
      const double2 b = row2[q], x = __ldg(rho2 + q);
      s = fma(b.x, x.x, s);
      s1 = fma(b.y, x.y, s1);
    }
    s += s1;
  } else {
    for (int P = lane; P < naux; P += 32) s = fma(row[P], __ldg(rho + P), s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    J[(long long)mu * nao + nu] = s;
    J[(long long)nu * nao + mu] = s;
  }
}

void j_gemv_f64(const double *B, long long ldb, int nao, int naux, const double *rho, double *J,
                const int *rowmap, cudaStream_t st) {
  const long long nrows = (long long)nao * (nao + 1) / 2;
  j_gemv_kernel<<<(unsigned)((nrows + 7) / 8), 256, 0, st>>>(B, ldb, nao, naux, rho, J, rowmap);
  DFJK_LAUNCHED();
}

// Bfull[(mu nao + nu) ldb + P] = Bc[rowmap[mu nao + nu] ldb + P] (0 where the
// map is -1): one block per (mu, nu) pair, threads along P (coalesced).
__global__ void __launch_bounds__(256) unpack_rows_kernel(const double *__restrict__ Bc, long long ldb, int nao,
                                                          const int *__restrict__ rowmap, double *__restrict__ Bf) {
  const long long e = blockIdx.x;  // mu nao + nu
  const int row = rowmap[e];
  double *dst = Bf + e * ldb;
  if (row < 0) {
    for (long long P = threadIdx.x; P < ldb; P += 256) dst[P] = 0.0;
    return;
  }
  const double *src = Bc + (long long)row * ldb;
  for (long long P = threadIdx.x; P < ldb; P += 256) dst[P] = src[P];
}

void unpack_rows_f64(const double *Bc, long long ldb, int nao, const int *rowmap, double *Bfull, cudaStream_t st) {
  const long long n2 = (long long)nao * nao;
  if (n2 == 0) return;
  unpack_rows_kernel<<<(unsigned)n2, 256, 0, st>>>(Bc, ldb, nao, rowmap, Bfull);
  DFJK_LAUNCHED();
}

// rowmap[mu nao + nu] = rowmap[nu nao + mu] = m for every column m with
// colmu[m] >= 0 (the map is -1 elsewhere).
__global__ void build_rowmap_kernel(const int *__restrict__ colmu, const int *__restrict__ colnu, long long ncol,
                                    int nao, int *__restrict__ rowmap) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ncol) return;
  const int mu = colmu[m], nu = colnu[m];
  if (mu < 0) return;
  rowmap[(long long)mu * nao + nu] = (int)m;
  rowmap[(long long)nu * nao + mu] = (int)m;
}

void build_rowmap(const int *colmu, const int *colnu, long long ncol, int nao, int *rowmap, cudaStream_t st) {
  DFJK_CUDA_CHECK(cudaMemsetAsync(rowmap, 0xFF, (size_t)nao * nao * sizeof(int), st));
  if (ncol == 0) return;
  build_rowmap_kernel<<<(unsigned)((ncol + 255) / 256), 256, 0, st>>>(colmu, colnu, ncol, nao, rowmap);
  DFJK_LAUNCHED();
}

// ---- reductions -----------------------------------------------------------------------

__global__ void reduce_sym_kernel(const double *__restrict__ part, int nsplit, int n,
                                  double *__restrict__ out, int add) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int mu = (int)(e / n), nu = (int)(e % n);
  if (nu > mu) return;
  double s = add ? out[e] : 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(long long)k * n * n + e];
  out[e] = s;
  out[(long long)nu * n + mu] = s;
}

void reduce_sym_f64(const double *part, int nsplit, int n, double *out, cudaStream_t st, int add) {
  const long long n2 = (long long)n * n;
  reduce_sym_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(part, nsplit, n, out, add);
  DFJK_LAUNCHED();
}

__global__ void mirror_lower_kernel(double *__restrict__ K, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int mu = (int)(e / n), nu = (int)(e % n);
  if (nu > mu) K[e] = K[(long long)nu * n + mu];
}

void mirror_lower_f64(double *K, int n, cudaStream_t st) {
  const long long n2 = (long long)n * n;
  mirror_lower_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(K, n);
  DFJK_LAUNCHED();
}

constexpr int EN_BLOCKS = 256;

__global__ void __launch_bounds__(256) energy_partial_kernel(const double *__restrict__ D,
                                                             const double *__restrict__ J,
                                                             const double *__restrict__ K,
                                                             long long n2, double *work) {
  __shared__ double sj[256], sk[256];
  double aj = 0.0, ak = 0.0;
  for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < n2; e += (long long)EN_BLOCKS * 256) {
    aj = fma(D[e], J[e], aj);
    ak = fma(D[e], K[e], ak);
  }
  sj[threadIdx.x] = aj;
  sk[threadIdx.x] = ak;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sj[threadIdx.x] += sj[threadIdx.x + s];
      sk[threadIdx.x] += sk[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    work[2 * blockIdx.x] = sj[0];
    work[2 * blockIdx.x + 1] = sk[0];
  }
}

__global__ void energy_final_kernel(const double *__restrict__ work, double *e) {
  __shared__ double sj[EN_BLOCKS], sk[EN_BLOCKS];
  sj[threadIdx.x] = work[2 * threadIdx.x];
  sk[threadIdx.x] = work[2 * threadIdx.x + 1];
  __syncthreads();
  for (int s = EN_BLOCKS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sj[threadIdx.x] += sj[threadIdx.x + s];
      sk[threadIdx.x] += sk[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    e[0] = 0.5 * sj[0];
    e[1] = 0.5 * sk[0];
  }
}

void energies_f64(const double *D, const double *J, const double *K, int n, double *e,
                  double *work, cudaStream_t st) {
  energy_partial_kernel<<<EN_BLOCKS, 256, 0, st>>>(D, J, K, (long long)n * n, work);
  DFJK_LAUNCHED();
  energy_final_kernel<<<1, EN_BLOCKS, 0, st>>>(work, e);
  DFJK_LAUNCHED();
}

__global__ void max_sqrt_diag_kernel(const double *V, int n, int ld, double *out) {
  __shared__ double s[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) m = fmax(m, sqrt(fmax(V[(long long)i * ld + i], 0.0)));
  s[threadIdx.x] = m;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

void max_sqrt_diag(const double *V, int n, int ld, double *out, cudaStream_t st) {
  max_sqrt_diag_kernel<<<1, 256, 0, st>>>(V, n, ld, out);
  DFJK_LAUNCHED();
}

__global__ void screen_kernel(const double *q, int n, const double *maxdiag, double thresh,
                              int *keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keep[i] = (q[i] * (*maxdiag) >= thresh) ? 1 : 0;
}

void screen_pairs(const double *q, int n, const double *maxdiag, double thresh, int *keep,
                  cudaStream_t st) {
  if (n == 0) return;
  screen_kernel<<<ceil_div(n, 256), 256, 0, st>>>(q, n, maxdiag, thresh, keep);
  DFJK_LAUNCHED();
}

__global__ void fill_kernel(double *p, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

void fill_f64(double *p, long long n, double v, cudaStream_t st) {
  if (n == 0) return;
  fill_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(p, n, v);
  DFJK_LAUNCHED();
}

__global__ void gather2d_kernel(const double *in, long long ldi, const int *pr, const int *pc,
                                int nr, int nc, double *out, long long ldo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nr * nc) return;
  const int i = (int)(e / nc), j = (int)(e % nc);
  out[i * ldo + j] = pr[i] < 0 ? 0.0 : in[(long long)pr[i] * ldi + pc[j]];
}

void gather2d_f64(const double *in, long long ldi, const int *perm_r, const int *perm_c, int nr,
                  int nc, double *out, long long ldo, cudaStream_t st) {
  const long long n = (long long)nr * nc;
  if (n == 0) return;
  gather2d_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, ldi, perm_r, perm_c, nr, nc, out, ldo);
  DFJK_LAUNCHED();
}

__global__ void gather_B_kernel(const double *Bint, long long ldb, int nao, const int *perm,
                                int naux, double *out, const int *rowmap) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n2 = (long long)nao * nao;
  if (e >= n2 * naux) return;
  const int P = (int)(e / n2);
  const long long mn = e % n2;
  const long long row = rowmap ? rowmap[mn] : mn;
  out[e] = row < 0 ? 0.0 : Bint[row * ldb + perm[P]];
}

void gather_B_f64(const double *Bint, long long ldb, int nao, const int *perm, int naux,
                  double *out, const int *rowmap, cudaStream_t st) {
  const long long n = (long long)nao * nao * naux;
  if (n == 0) return;
  gather_B_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Bint, ldb, nao, perm, naux, out, rowmap);
  DFJK_LAUNCHED();
}

}  // namespace dfjk
