// Exact sliced-product GEMM on the tcgen05 tensor cores (ozaki.cu).
//
// An FP64 operand row is split, per block of OZ_KB consecutive K elements,
// into S integer "slices" of 6 bits under a common power-of-two exponent e:
//     x = 2^e * sum_{s<S} a_s 2^{-6(s+1)},  a_0 in [-64, 64], a_s in [-32, 31],
// each a_s stored exactly as BF16.  A product of two slices is an integer
// below 2^12 and a K-block sum of them stays below 2^24, so the FP32 tensor
// core accumulation is exact whatever its internal rounding.  Products with
// s + t = l share TMEM accumulator l; levels l < S are kept (error about
// 2^-6S of |A||B| per term), combined exactly in int64 and added to FP64
// accumulators once per K-block with scale 2^(eA + eB).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dfjk {

constexpr int OZ_W = 6;      // bits per slice
constexpr int OZ_KB = 1024;  // K elements per exponent block
constexpr int OZ_BM = 128, OZ_BN = 64;
constexpr int OZ_BK = 32;   // K pitch granularity of the slice planes

// Slices of an operand: planes [batch][S][rows_pad][kpitch] (BF16, K
// contiguous) and exponents [batch][rows_pad][nkb] (int32).
// Layout of data: [batch][S][rows_pad][kpitch], or, for long K (kblk = 1,
// more than 4 exponent blocks), K-blocked [batch][S][nkb][rows_pad][1024] so
// that the rows of one TMA box lie 2 KB apart instead of a whole K row apart
// (a box of the K GEMM's X slices would otherwise touch 128 pages).
struct SlicedOp {
  __nv_bfloat16 *data = nullptr;
  int *expo = nullptr;
  int batch = 1, S = 0, rows = 0, rows_pad = 0, K = 0, kpitch = 0, nkb = 0, kblk = 0, row_tile = 0;
  size_t bytes() const {
    return (size_t)batch * S * rows_pad * kpitch * 2 + (size_t)batch * rows_pad * nkb * 4;
  }
};

// Sizes an operand (rows padded to `row_tile`, K pitch to OZ_BK) and allocates it.
void oz_alloc(SlicedOp &op, int batch, int S, int rows, int K, int row_tile);
void oz_free(SlicedOp &op);
// A view of op's buffers sized for `rows` rows and K columns (at most the
// allocated rows and K): the layout a fresh allocation of that size would
// have, placed at the start of op's buffers.  Used for the short last chunk
// of a chunked reduction without reallocating.
SlicedOp oz_view(const SlicedOp &op, int rows, int K);

// Fills `op` from the FP64 view x(z, r, k) = src[z sz + r sr + k sk]
// (rows >= op.rows and k >= op.K are zero).
// rows_per_block: rows of a row-contiguous source per block of the fused
// slicing kernel (8, 16 or 32; 0 = the default, 16, or DFJK_SLICE_ROWS).
void oz_slice_f64(const double *src, long long sz, long long sr, long long sk, SlicedOp &op,
                  cudaStream_t st, int rows_per_block = 0);

struct OzGemmArgs {
  int M = 0, N = 0, K = 0;
  int nz = 1;            // grid z: batches, or split-K parts
  int a_batched = 0;     // A indexed by z
  int b_batched = 0;     // B indexed by z
  int kb_per_split = 0;  // >0: z selects K-blocks [z kb_per_split, (z+1) kb_per_split)
  int k_upto_n = 0;      // K limited to < end of the N tile (B lower triangular)
  int lower_only = 0;    // skip tiles strictly above the diagonal
  int mode = 0;          // 0: out[z out_bs + m ldo + n] = C;
                         // 2: split-K in order, out[m ldo + n] (+)= C of split z
                         //    after splits 0..z-1 (persistent kernel only)
  int *tile_seq = nullptr;  // mode 2: per (tile, drain warp) split counters
  int accumulate = 0;    // mode 2: split 0 also adds onto out (a later chunk of
                         // the reduction range, in chunk order)
  double *out = nullptr;
  long long ldo = 0, out_bs = 0;
  int *status = nullptr;       // STATUS_TIMEOUT on an expired wait
  long long timeout = 1 << 26; // polls per mbarrier wait
  int phase = -1;              // phase timer id of this launch (-1: none)
  int *tile_ctr = nullptr;     // device int for the dynamic tile queue; oz_gemm
                               // zeroes it on the stream, so launches that can
                               // run concurrently need distinct counters
};

// B stored by rows of ldb doubles (P contiguous), one row per kept AO pair:
// rowmap[mu nao + nu] = rowmap[nu nao + mu] is the row of pair (mu, nu), -1 for
// a screened pair (B is zero there).  Its slices for the X GEMM are batch mu,
// rows P, K nu, with one exponent per (mu, P, 1024-block of nu).  Both
// functions below read each stored row once (32 x 32 tiles of the mu >= nu
// pair triangle, each written for batch mu and for batch nu) and skip the
// screened pairs.

// The exponents for every mu and the rows P < pre_rows (rows np..pre_rows-1
// get 0): expo[(mu pre_rows + P) nkb + kb].  B does not change between
// builds, so a handle computes them once.
void oz_expo_packed(const double *B, long long ldb, const int *rowmap, int nao, int np, int pre_rows, int *expo,
                    cudaStream_t st);
// The slices of the chunk of rows P [p0, p0 + op.rows) for all mu (batch = K
// = nao), with the exponents from `pre` (oz_expo_packed), which are also
// copied into op.expo.  p0 % 32 == 0 and p0 + op.rows_pad <= pre_rows.
// rows_per_block: rows P per block (4, 8 or 16; 0 = the default, 4, or
// DFJK_PSLICE_ROWS).
void oz_slice_f64_packed_pre(const double *B, long long ldb, const int *rowmap, const int *pre, int pre_rows, int p0,
                             SlicedOp &op, cudaStream_t st, int rows_per_block = 0);

// True when DFJK_OZ_SIMPLE=1 selects the one-tile-per-CTA kernel (no mode 2).
bool oz_simple_mode();
// Counters mode 2 needs for a launch of M x N (ints).
size_t oz_tile_seq_count(int M, int N);

// out = A B^T with A (M x K) and B (N x K) in sliced form, both with S slices.
void oz_gemm(const SlicedOp &A, const SlicedOp &B, const OzGemmArgs &g, cudaStream_t st);

}  // namespace dfjk
