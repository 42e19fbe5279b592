// Exact sliced-product GEMM on tcgen05 tensor cores, and the slicing kernels
// that feed it.  See ozaki.cuh for the representation.  The scheme follows the
// error-free splitting idea of Ozaki et al. (Numer. Algorithms 59, 2012):
// split each operand into pieces whose products and partial sums are exact in
// the accumulator, and recombine in higher precision.  Here the pieces are
// 6-bit integers in BF16, the accumulator is FP32 in TMEM, the recombination
// int64 + FP64 in registers.
//
// Kernel layout (one CTA per SM: 512 TMEM columns, ~200 KB shared memory):
//   tile 128 (M, one TMEM lane per row) x 64 (N) ; K stages of 16 (32-byte
//   swizzled rows) ; 4-5 stage TMA ring ; one thread issues TMA, one MMA ;
//   S level accumulators of 64 TMEM columns, filled two levels per MMA
//   (oz_mma_step) ; after each K-block of 1024 the epilogue drains every TMEM
//   row: level sums -> int64 -> FP64 register accumulators.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "ozaki.cuh"
#include "pool.cuh"
#include "tc.cuh"

namespace dfjk {

// ---- slicing --------------------------------------------------------------------

__device__ __forceinline__ int oz_expo_of(double mx) {
  if (!(mx > 0.0)) return 0;
  const long long u = __double_as_longlong(mx);
  const int ex = (int)((u >> 52) & 0x7FF);
  return ex == 0 ? -1021 : ex - 1022;  // |x| <= mx < 2^e
}

// round(x 2^(6S - e)) as an integer, |result| <= 2^(6S).
template <int S>
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const long long u = __double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero (subnormals are far below any row maximum here)
  const long long mant = (u & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = ex - 1075 + 6 * S - e;
  long long n;
  if (sh >= 0) n = mant << sh;
  else if (sh < -60) n = 0;
  else n = (mant + (1LL << (-sh - 1))) >> (-sh);
  return u < 0 ? -n : n;
}

// The S balanced base-64 digits of n (|n| <= 2^(6S)), n = sum_s d_s
// 64^(S-1-s) with d_s in [-32, 31] for s >= 1, as FP32 bit patterns whose
// high halves are the digits' BF16 patterns.  Adding 32 (1 + 64 + ... +
// 64^(S-2)) turns the low S - 1 digits into plain 6-bit fields u_s = d_s + 32
// and leaves d_0 in the top bits; a digit becomes an exact float through the
// 1.5 2^23 bias (an integer add into the mantissa and one FP32 subtract), so
// no conversion instructions are needed.
template <int S>
__device__ __forceinline__ void oz_digits(long long n, uint32_t (&f)[S]) {
  constexpr long long C = 32 * (((1LL << (6 * (S - 1))) - 1) / 63);
  const long long m = n + C;
  const unsigned long long um = (unsigned long long)m;
  f[0] = __float_as_uint(__int_as_float(0x4B400000 + (int)(m >> (6 * (S - 1)))) - 12582912.0f);
#pragma unroll
  for (int s = 1; s < S; ++s) {
    const uint32_t u = (uint32_t)(um >> (6 * (S - 1 - s))) & 63u;
    f[s] = __float_as_uint(__uint_as_float(0x4B400000u + u) - 12582944.0f);
  }
}
__device__ __forceinline__ __nv_bfloat16 oz_bf16_of(uint32_t fbits) {
  return __ushort_as_bfloat16((unsigned short)(fbits >> 16));
}
// Two digits' FP32 patterns -> one word of two BF16 (a at the lower address).
__device__ __forceinline__ uint32_t oz_pack2(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// Element offset of slice s of (z, r, k) in a SlicedOp's data (k % 8 == 0 for
// the 16-byte stores below, which then stay inside one 1024-wide K block).
__device__ __forceinline__ long long oz_off(int z, int s, int r, int k, int S, int rows_pad, int kpitch,
                                            int nkb, int kblk) {
  if (kblk) return ((((long long)z * S + s) * nkb + (k >> 10)) * rows_pad + r) * OZ_KB + (k & (OZ_KB - 1));
  return (((long long)z * S + s) * rows_pad + r) * kpitch + k;
}

// Exponent of every (z, row, K-block); one warp per entry, lanes along K
// (for K-contiguous sources).
__global__ void oz_expo_warp_kernel(const double *__restrict__ src, long long sz, long long sr,
                                    long long sk, int batch, int rows, int K, int rows_pad, int nkb,
                                    int *__restrict__ expo) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)batch * rows_pad * nkb) return;
  const int kb = (int)(w % nkb);
  const int r = (int)((w / nkb) % rows_pad);
  const int z = (int)(w / ((long long)nkb * rows_pad));
  double mx = 0.0;
  if (r < rows) {
    const int k1 = min(K, (kb + 1) * OZ_KB);
    const double *p = src + z * sz + r * sr;
    for (int k = kb * OZ_KB + lane; k < k1; k += 32) mx = fmax(mx, fabs(p[k * sk]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) expo[w] = oz_expo_of(mx);
}

// Same, one thread per entry walking K (for row-contiguous sources).
__global__ void oz_expo_thread_kernel(const double *__restrict__ src, long long sz, long long sr,
                                      long long sk, int batch, int rows, int K, int rows_pad, int nkb,
                                      int *__restrict__ expo) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)batch * rows_pad * nkb) return;
  const int r = (int)(t % rows_pad);
  const int kb = (int)((t / rows_pad) % nkb);
  const int z = (int)(t / ((long long)rows_pad * nkb));
  double mx = 0.0;
  if (r < rows) {
    const int k1 = min(K, (kb + 1) * OZ_KB);
    const double *p = src + z * sz + r * sr;
    for (int k = kb * OZ_KB; k < k1; ++k) mx = fmax(mx, fabs(p[k * sk]));
  }
  expo[((long long)z * rows_pad + r) * nkb + kb] = oz_expo_of(mx);
}

// Slices of 8 consecutive K elements of one row per thread.  `row_fast`
// selects the thread order (consecutive rows for row-contiguous sources).
template <int S>
__global__ void oz_slice_kernel(const double *__restrict__ src, long long sz, long long sr, long long sk,
                                int batch, int rows, int K, int rows_pad, int kpitch, int nkb,
                                const int *__restrict__ expo, __nv_bfloat16 *__restrict__ out,
                                int row_fast, int kblk) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nkc = kpitch / 8;
  if (t >= (long long)batch * rows_pad * nkc) return;
  int z, r, kc;
  if (row_fast) {
    r = (int)(t % rows_pad);
    kc = (int)((t / rows_pad) % nkc);
    z = (int)(t / ((long long)rows_pad * nkc));
  } else {
    kc = (int)(t % nkc);
    r = (int)((t / nkc) % rows_pad);
    z = (int)(t / ((long long)rows_pad * nkc));
  }
  const int k0 = kc * 8;
  const int e = expo[((long long)z * rows_pad + r) * nkb + k0 / OZ_KB];
  uint32_t w[S][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = k0 + j;
    const double x = (r < rows && k < K) ? src[z * sz + r * sr + (long long)k * sk] : 0.0;
    uint32_t f[S];
    oz_digits<S>(oz_fixed<S>(x, e), f);
#pragma unroll
    for (int s = 0; s < S; ++s) w[s][j / 2] = (j & 1) ? oz_pack2(w[s][j / 2], f[s]) : f[s];
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
    *reinterpret_cast<uint4 *>(out + oz_off(z, s, r, k0, S, rows_pad, kpitch, nkb, kblk)) =
        make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// Slices of a 64 (rows) x 64 (K) tile per block for row-contiguous sources:
// reads coalesced along rows, digits staged in shared memory as [s][row][k],
// written as 128-byte row segments along K.
template <int S>
__global__ void __launch_bounds__(256) oz_slice_tr_kernel(const double *__restrict__ src, long long sz,
                                                          long long sk, int rows, int K, int rows_pad,
                                                          int kpitch, int nkb, const int *__restrict__ expo,
                                                          __nv_bfloat16 *__restrict__ out, int kblk) {
  extern __shared__ __nv_bfloat16 tile[];  // [S][64][64 + 8]
  constexpr int LD = 72;
  const int z = blockIdx.z, r0 = blockIdx.y * 64, k0 = blockIdx.x * 64;
  const int rr = threadIdx.x & 63, kq = threadIdx.x >> 6;
  const int r = r0 + rr;
  const int e = expo[((long long)z * rows_pad + r) * nkb + k0 / OZ_KB];
  for (int kk = kq; kk < 64; kk += 4) {
    const int k = k0 + kk;
    const double x = (r < rows && k < K) ? src[z * sz + r + (long long)k * sk] : 0.0;
    uint32_t f[S];
    oz_digits<S>(oz_fixed<S>(x, e), f);
#pragma unroll
    for (int s = 0; s < S; ++s) tile[(s * 64 + rr) * LD + kk] = oz_bf16_of(f[s]);
  }
  __syncthreads();
  const int c8 = threadIdx.x & 7, rw = threadIdx.x >> 3;  // 8 x 16-byte chunks per row
#pragma unroll
  for (int s = 0; s < S; ++s)
    for (int rb = rw; rb < 64; rb += 32) {
      const int kc = k0 + c8 * 8;
      if (kc < kpitch) {
        const uint4 v = *reinterpret_cast<const uint4 *>(&tile[(s * 64 + rb) * LD + c8 * 8]);
        *reinterpret_cast<uint4 *>(out + oz_off(z, s, r0 + rb, kc, S, rows_pad, kpitch, nkb, kblk)) = v;
      }
    }
}

// Row-contiguous sources, exponents and slices in one kernel: a block owns R
// rows of one batch and walks all of K twice, first for the per-(row, K-block)
// maxima, then for the slices.  R rows x K doubles per block (58 KB for R = 8
// and K = 900) keeps the second read in L2 with every SM's blocks in flight;
// lanes run along the rows (8 R contiguous bytes per K index).
template <int S, int R = 8>
__global__ void __launch_bounds__(256) oz_slice_tr_fused_kernel(const double *__restrict__ src, long long sz,
                                                                long long sk, int rows, int K, int rows_pad,
                                                                int kpitch, int nkb, int *__restrict__ expo,
                                                                __nv_bfloat16 *__restrict__ out, int kblk) {
  // slices staged K-major, [s][k][row] with R + 1 elements per k: the writes
  // (lanes along rows) and the reads of 8 consecutive k of one row (lanes
  // along k chunks) both spread over the shared-memory banks
  constexpr int KG = 256 / R, LDK = R + 1, MAXKB = 8;
  __shared__ __nv_bfloat16 tile[S * 64 * LDK];
  __shared__ unsigned long long rmax[R][MAXKB];
  __shared__ int rexp[R][MAXKB];
  const int z = blockIdx.y, r0 = blockIdx.x * R;
  const int rr = threadIdx.x % R, kq = threadIdx.x / R;  // KG groups along K
  const int r = r0 + rr;
  const bool live = r < rows;
  auto at = [&](int k) -> double { return src[z * sz + (long long)k * sk + r]; };
  if (threadIdx.x < R * MAXKB) rmax[threadIdx.x / MAXKB][threadIdx.x % MAXKB] = 0ull;
  __syncthreads();
  // pass 1: |x| maxima per K block, on the bit patterns (non-negative doubles
  // order like their bits)
  for (int kb = 0; kb < nkb; ++kb) {
    unsigned long long mx = 0;
    if (live) {
      const int k1 = min(K, (kb + 1) * OZ_KB);
#pragma unroll 4
      for (int k = kb * OZ_KB + kq; k < k1; k += KG)
        mx = max(mx, (unsigned long long)__double_as_longlong(at(k)) & 0x7FFFFFFFFFFFFFFFull);
    }
    // lanes with the same row in a warp (32 / R of them)
#pragma unroll
    for (int o = R; o < 32; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) < R) atomicMax(&rmax[rr][kb], mx);
  }
  __syncthreads();
  if (threadIdx.x < R * nkb) {
    const int q = threadIdx.x / nkb, kb = threadIdx.x % nkb;
    const int e = oz_expo_of(__longlong_as_double((long long)rmax[q][kb]));
    rexp[q][kb] = e;
    expo[((long long)z * rows_pad + r0 + q) * nkb + kb] = e;
  }
  __syncthreads();
  // pass 2: slices, 64 K at a time, staged [s][row][k] and written along K
  for (int k0 = 0; k0 < kpitch; k0 += 64) {
    const int e = rexp[rr][k0 / OZ_KB];
    for (int kk = kq; kk < 64; kk += KG) {
      const int k = k0 + kk;
      const double x = (live && k < K) ? at(k) : 0.0;
      uint32_t f[S];
      oz_digits<S>(oz_fixed<S>(x, e), f);
#pragma unroll
      for (int s = 0; s < S; ++s) tile[(s * 64 + kk) * LDK + rr] = oz_bf16_of(f[s]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * R * 8; i += 256) {  // (slice, row, chunk of 8 K)
      const int s = i / (R * 8), rw = (i / 8) % R, c8 = i % 8;
      const int kc = k0 + c8 * 8;
      if (kc < kpitch) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = tile[(s * 64 + c8 * 8 + t) * LDK + rw];
        *reinterpret_cast<uint4 *>(out + oz_off(z, s, r0 + rw, kc, S, rows_pad, kpitch, nkb, kblk)) =
            *reinterpret_cast<const uint4 *>(v);
      }
    }
    __syncthreads();
  }
}

// Slicing of B (rows of the kept AO pairs, found through rowmap) reading each
// stored row once.
// A block owns a 32 x 32 tile of the pair triangle (mu block >= nu block) and
// R rows P, and stages the tile's FP64 values in shared memory (pairs with
// mu < nu on the diagonal tiles are read from (nu, mu)); consecutive pairs of
// one mu are rows of B ldb doubles apart, R contiguous doubles each.
// MODE 2: writes the slices of batch mu at K index nu and, off the diagonal,
// of batch nu at K index mu, with exponents from `pre`; tiles beyond nao (up
// to the K pitch) write the zero padding.  MODE 1: per (mu, P, 1024-block of
// nu) maxima of |x|, folded across tiles with atomicMax on the encoded
// exponent (0 for an all-zero block, else exponent + OZ_EXPO_BIAS; larger
// |x| never has a smaller exponent).
constexpr int OZ_EXPO_BIAS = 4096;
constexpr int OZ_TT = 32;  // tile edge in AO indices

__host__ __device__ constexpr int oz_sym_smem(int R) {
  return OZ_TT * OZ_TT * (R + 1) * 8 + 2 * OZ_TT * R * 4 + OZ_TT * OZ_TT * 4;
}

template <int R, int MODE>
__global__ void __launch_bounds__(256) oz_slice_sym_kernel(const double *__restrict__ B, long long ldb,
                                                           const int *__restrict__ rowmap, int nao, int rows,
                                                           int p0, int rows_pad, int kpitch, int nkb, int kblk,
                                                           const int *__restrict__ pre, int pre_rows,
                                                           int *__restrict__ expo_out, __nv_bfloat16 *__restrict__ out) {
  constexpr int RP = R + 1;
  extern __shared__ __align__(16) uint8_t sym_smem[];
  double *tile = reinterpret_cast<double *>(sym_smem);  // [mu_l][nu_l][P], P stride 1, nu stride RP
  int *eD = reinterpret_cast<int *>(tile + OZ_TT * OZ_TT * RP);  // [mu_l][P]: batch mu, K block of nu0
  int *eT = eD + OZ_TT * R;                                    // [nu_l][P]: batch nu, K block of mu0
  int *tmap = eT + OZ_TT * R;                                  // [mu_l][nu_l]: row of B, -1 if none
  // grid x: row groups (fastest, so that the blocks reading the neighbouring
  // rows of one pair run together and share its cache lines); grid y: tile
  // t of the lower triangle -> (ti >= tj)
  const long long t = blockIdx.y;
  int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while ((long long)ti * (ti + 1) / 2 > t) --ti;
  const int tj = (int)(t - (long long)ti * (ti + 1) / 2);
  const int mu0 = ti * OZ_TT, nu0 = tj * OZ_TT, r0 = blockIdx.x * R;
  const bool diag = ti == tj;
  // the tile's rows of B (one load per pair, 32 consecutive nu per mu), so
  // that the loads of B below do not wait on the map
  bool any = false;
  for (int q = threadIdx.x; q < OZ_TT * OZ_TT; q += 256) {
    const int mu = mu0 + q / OZ_TT, nu = nu0 + q % OZ_TT;
    const int row = (mu < nao && nu < nao) ? rowmap[(long long)mu * nao + nu] : -1;
    tmap[q] = row;
    any |= row >= 0;
  }
  any = __syncthreads_or(any);
  if (MODE == 1 && !any) return;  // every pair of the tile screened: maxima 0
  // stage the tile: R lanes per pair, 256 / R pairs per pass, 16 loads in
  // flight per thread
  constexpr int PER = OZ_TT * OZ_TT * R / 256, UN = PER < 16 ? PER : 16;
  static_assert(PER % UN == 0, "tile loads");
#pragma unroll 1
  for (int u0 = 0; u0 < PER; u0 += UN) {
    double v[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int i = threadIdx.x + (u0 + u) * 256;
      const int P = i % R, q = i / R, r = r0 + P;
      const int row = tmap[q];
      v[u] = (row >= 0 && r < rows) ? B[(long long)row * ldb + p0 + r] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int i = threadIdx.x + (u0 + u) * 256;
      tile[((i / R) / OZ_TT * OZ_TT + (i / R) % OZ_TT) * RP + i % R] = v[u];
    }
  }
  if (MODE == 2) {
    for (int i = threadIdx.x; i < 2 * OZ_TT * R; i += 256) {
      const int P = i % R, l = (i / R) % OZ_TT, tr = i / (OZ_TT * R);
      const int z = (tr ? nu0 : mu0) + l, kb = (tr ? mu0 : nu0) >> 10;
      (tr ? eT : eD)[l * R + P] = z < nao ? pre[((long long)z * pre_rows + p0 + r0 + P) * nkb + kb] : 0;
    }
  }
  __syncthreads();
  if constexpr (MODE == 1) {
    // thread (l, P): direct maximum over nu of row mu0 + l; transposed over mu of column nu0 + l
    for (int i = threadIdx.x; i < 2 * OZ_TT * R; i += 256) {
      const int P = i % R, l = (i / R) % OZ_TT, tr = i / (OZ_TT * R);
      if (tr && diag) continue;
      const int z = (tr ? nu0 : mu0) + l, kb = (tr ? mu0 : nu0) >> 10;
      if (z >= nao) continue;
      // maxima of the high words of |x| (sign cleared): the exponent lives
      // there and non-negative doubles order like their bits, so 32-bit
      // integer maxima suffice (values whose high word is 0, below 2^-1042,
      // count as zero)
      unsigned int mx = 0;
#pragma unroll 8
      for (int o = 0; o < OZ_TT; ++o) {
        const double x = tr ? tile[(o * OZ_TT + l) * RP + P] : tile[(l * OZ_TT + o) * RP + P];
        mx = max(mx, (unsigned int)__double2hiint(x) & 0x7FFFFFFFu);
      }
      if (mx) {
        const int ex = (int)(mx >> 20);  // biased exponent, as oz_expo_of takes it
        atomicMax(expo_out + ((long long)z * pre_rows + r0 + P) * nkb + kb,
                  (ex == 0 ? -1021 : ex - 1022) + OZ_EXPO_BIAS);
      }
    }
    return;
  } else {
  // slices: item (l, P, g) = 8 consecutive K of batch mu0 + l (direct) or nu0 + l
  // (transposed), one 16-byte store per slice; 4 lanes cover 32 K (64 bytes)
  for (int i = threadIdx.x; i < 2 * OZ_TT * R * 4; i += 256) {
    const int g = i % 4, P = (i / 4) % R, l = (i / (4 * R)) % OZ_TT, tr = i / (4 * R * OZ_TT);
    if (tr && diag) break;  // the transposed half comes last
    const int z = (tr ? nu0 : mu0) + l;
    if (z >= nao) continue;
    const int e = (tr ? eT : eD)[l * R + P];
    const int k = (tr ? mu0 : nu0) + g * 8;
    uint32_t w[6][4];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int o = g * 8 + u;
      uint32_t f[6];
      oz_digits<6>(oz_fixed<6>(tr ? tile[(o * OZ_TT + l) * RP + P] : tile[(l * OZ_TT + o) * RP + P], e), f);
#pragma unroll
      for (int sl = 0; sl < 6; ++sl) w[sl][u / 2] = (u & 1) ? oz_pack2(w[sl][u / 2], f[sl]) : f[sl];
    }
#pragma unroll
    for (int sl = 0; sl < 6; ++sl)
      *reinterpret_cast<uint4 *>(out + oz_off(z, sl, r0 + P, k, 6, rows_pad, kpitch, nkb, kblk)) =
          make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
  }
  }
}

// expo[i] encoded as above -> exponent
__global__ void oz_expo_decode_kernel(int *expo, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) expo[i] = expo[i] ? expo[i] - OZ_EXPO_BIAS : 0;
}

template <int R, int MODE>
static void launch_oz_sym(dim3 grid, const double *B, long long ldb, const int *rowmap, int nao, int rows, int p0,
                          int rows_pad, int kpitch, int nkb, int kblk, const int *pre, int pre_rows, int *expo_out,
                          __nv_bfloat16 *out, cudaStream_t st) {
  constexpr int SM = oz_sym_smem(R);
  static bool attr_set = false;
  if (!attr_set) {
    DFJK_CUDA_CHECK(cudaFuncSetAttribute(oz_slice_sym_kernel<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM));
    attr_set = true;
  }
  oz_slice_sym_kernel<R, MODE><<<grid, 256, SM, st>>>(B, ldb, rowmap, nao, rows, p0, rows_pad, kpitch, nkb, kblk,
                                                       pre, pre_rows, expo_out, out);
  DFJK_LAUNCHED();
}

static void oz_shape(SlicedOp &op, int batch, int S, int rows, int K, int row_tile) {
  op.batch = batch;
  op.S = S;
  op.rows = rows;
  op.row_tile = row_tile;
  op.rows_pad = ((rows + row_tile - 1) / row_tile) * row_tile;
  op.K = K;
  op.nkb = (K + OZ_KB - 1) / OZ_KB;
  op.kblk = op.nkb > 4 ? 1 : 0;
  op.kpitch = op.kblk ? op.nkb * OZ_KB : ((K + OZ_BK - 1) / OZ_BK) * OZ_BK;
}

SlicedOp oz_view(const SlicedOp &op, int rows, int K) {
  if (rows > op.rows || K > op.K || rows < 1 || K < 1) throw Error{DFJK_ERR_ARG, "oz_view: larger than the buffer"};
  SlicedOp v;
  oz_shape(v, op.batch, op.S, rows, K, op.row_tile);
  v.data = op.data;
  v.expo = op.expo;
  return v;
}

void oz_alloc(SlicedOp &op, int batch, int S, int rows, int K, int row_tile) {
  oz_free(op);
  oz_shape(op, batch, S, rows, K, row_tile);
  const size_t nd = (size_t)batch * S * op.rows_pad * op.kpitch;
  const size_t ne = (size_t)batch * op.rows_pad * op.nkb;
  op.data = (__nv_bfloat16 *)pool_alloc(nd * sizeof(__nv_bfloat16));
  try {
    op.expo = (int *)pool_alloc(ne * sizeof(int));
  } catch (...) {
    pool_free(op.data, nd * sizeof(__nv_bfloat16));
    op.data = nullptr;
    throw;
  }
}

void oz_free(SlicedOp &op) {
  if (op.data) pool_free(op.data, (size_t)op.batch * op.S * op.rows_pad * op.kpitch * sizeof(__nv_bfloat16));
  if (op.expo) pool_free(op.expo, (size_t)op.batch * op.rows_pad * op.nkb * sizeof(int));
  op.data = nullptr;
  op.expo = nullptr;
}

void oz_expo_packed(const double *B, long long ldb, const int *rowmap, int nao, int np, int pre_rows, int *expo,
                    cudaStream_t st) {
  const int nkb = (nao + OZ_KB - 1) / OZ_KB;
  if (pre_rows % 32 != 0 || pre_rows < np || nkb > 8 || np > ldb)
    throw Error{DFJK_ERR_UNSUPPORTED, "packed exponents: K <= 8192"};
  const long long n = (long long)nao * pre_rows * nkb;
  DFJK_CUDA_CHECK(cudaMemsetAsync(expo, 0, n * sizeof(int), st));
  const long long nb = (nao + OZ_TT - 1) / OZ_TT, tiles = nb * (nb + 1) / 2;
  if (tiles > 65535) throw Error{DFJK_ERR_ARG, "packed exponents: grid"};
  // 4 rows P per block: 46 KB of shared memory, 4 blocks per SM (8 rows: 80 KB,
  // 2 blocks, latency-bound)
  launch_oz_sym<4, 1>(dim3((unsigned)(pre_rows / 4), (unsigned)tiles), B, ldb, rowmap, nao, np, 0, 0, 0, nkb, 0,
                      nullptr, pre_rows, expo, nullptr, st);
  oz_expo_decode_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(expo, n);
  DFJK_LAUNCHED();
}

void oz_slice_f64_packed_pre(const double *B, long long ldb, const int *rowmap, const int *pre, int pre_rows, int p0,
                             SlicedOp &op, cudaStream_t st, int rows_per_block) {
  // every row a block touches, padding included, has a precomputed exponent;
  // batch = nao, K = nao
  if (op.S != 6 || op.rows_pad % 32 != 0 || op.nkb > 8 || p0 % 32 != 0 || p0 + op.rows_pad > pre_rows ||
      op.batch != op.K || op.kpitch % OZ_TT != 0 || p0 + op.rows > ldb)
    throw Error{DFJK_ERR_UNSUPPORTED, "packed slicing: 6 slices, K <= 8192, exponent rows"};
  // rows P per block: 4 (default: 4 blocks per SM; 8 rows fit 2 and were
  // latency-bound, 2.36 against 1.96 ms per 60-atom chunk), 8 or 16
  // (DFJK_PSLICE_ROWS or the tuning table)
  static const int R_env = [] {
    const char *e = std::getenv("DFJK_PSLICE_ROWS");
    const int v = e ? std::atoi(e) : 4;
    return (v == 8 || v == 16) ? v : 4;
  }();
  const int R = (rows_per_block == 4 || rows_per_block == 8 || rows_per_block == 16) ? rows_per_block : R_env;
  // exponents of the chunk's rows, copied for the GEMM
  DFJK_CUDA_CHECK(cudaMemcpy2DAsync(op.expo, (size_t)op.rows_pad * op.nkb * sizeof(int), pre + (size_t)p0 * op.nkb,
                                    (size_t)pre_rows * op.nkb * sizeof(int), (size_t)op.rows_pad * op.nkb * sizeof(int),
                                    (size_t)op.batch, cudaMemcpyDeviceToDevice, st));
  const long long nb = op.kpitch / OZ_TT, tiles = nb * (nb + 1) / 2;
  if (tiles > 65535) throw Error{DFJK_ERR_ARG, "packed slicing: grid"};
  const dim3 grid((unsigned)(op.rows_pad / R), (unsigned)tiles);
  if (R == 4)
    launch_oz_sym<4, 2>(grid, B, ldb, rowmap, op.batch, op.rows, p0, op.rows_pad, op.kpitch, op.nkb, op.kblk, pre, pre_rows,
                        nullptr, op.data, st);
  else if (R == 16)
    launch_oz_sym<16, 2>(grid, B, ldb, rowmap, op.batch, op.rows, p0, op.rows_pad, op.kpitch, op.nkb, op.kblk, pre, pre_rows,
                         nullptr, op.data, st);
  else
    launch_oz_sym<8, 2>(grid, B, ldb, rowmap, op.batch, op.rows, p0, op.rows_pad, op.kpitch, op.nkb, op.kblk, pre, pre_rows,
                        nullptr, op.data, st);
}

void oz_slice_f64(const double *src, long long sz, long long sr, long long sk, SlicedOp &op,
                  cudaStream_t st, int rows_req) {
  if (sr == 1 && op.rows_pad % 8 == 0 && op.nkb <= 8) {
    // row-contiguous source: exponents and slices fused, one read from HBM;
    // rows per block 16 (measured best of 8 / 16 / 32 at 60 atoms; the
    // DFJK_SLICE_ROWS environment variable selects another)
    static const int rows_env = [] {
      const char *e = std::getenv("DFJK_SLICE_ROWS");
      const int v = e ? std::atoi(e) : 16;
      return (v == 8 || v == 32) ? v : 16;
    }();
    const int rows_per_block = (rows_req == 8 || rows_req == 16 || rows_req == 32) ? rows_req : rows_env;
    const int R = (op.rows_pad % rows_per_block == 0) ? rows_per_block : 8;
    dim3 grid((unsigned)(op.rows_pad / R), (unsigned)op.batch);
#define OZ_FUSED(SS, RR)                                                                                      \
  oz_slice_tr_fused_kernel<SS, RR><<<grid, 256, 0, st>>>(src, sz, sk, op.rows, op.K, op.rows_pad, op.kpitch,   \
                                                          op.nkb, op.expo, op.data, op.kblk)
    if (op.S == 6) {
      if (R == 32) OZ_FUSED(6, 32);
      else if (R == 16) OZ_FUSED(6, 16);
      else OZ_FUSED(6, 8);
    } else if (op.S == 8) {
      if (R == 32) OZ_FUSED(8, 32);
      else if (R == 16) OZ_FUSED(8, 16);
      else OZ_FUSED(8, 8);
    } else {
      throw Error{DFJK_ERR_UNSUPPORTED, "slice count must be 6 or 8"};
    }
#undef OZ_FUSED
    DFJK_LAUNCHED();
    return;
  }
  const long long nexp = (long long)op.batch * op.rows_pad * op.nkb;
  if (sk == 1) {
    oz_expo_warp_kernel<<<(unsigned)((nexp * 32 + 255) / 256), 256, 0, st>>>(
        src, sz, sr, sk, op.batch, op.rows, op.K, op.rows_pad, op.nkb, op.expo);
  } else {
    oz_expo_thread_kernel<<<(unsigned)((nexp + 255) / 256), 256, 0, st>>>(
        src, sz, sr, sk, op.batch, op.rows, op.K, op.rows_pad, op.nkb, op.expo);
  }
  DFJK_LAUNCHED();
  if (sr == 1 && op.rows_pad % 64 == 0) {
    // row-contiguous source: transpose through shared memory
    const size_t smem = (size_t)op.S * 64 * 72 * sizeof(__nv_bfloat16);
    dim3 grid((unsigned)((op.kpitch + 63) / 64), (unsigned)(op.rows_pad / 64), (unsigned)op.batch);
    static bool attr6 = false, attr8 = false;
    switch (op.S) {
      case 6:
        if (!attr6) {
          DFJK_CUDA_CHECK(cudaFuncSetAttribute(oz_slice_tr_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr6 = true;
        }
        oz_slice_tr_kernel<6><<<grid, 256, smem, st>>>(src, sz, sk, op.rows, op.K, op.rows_pad, op.kpitch,
                                                       op.nkb, op.expo, op.data, op.kblk);
        break;
      case 8:
        if (!attr8) {
          DFJK_CUDA_CHECK(cudaFuncSetAttribute(oz_slice_tr_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          attr8 = true;
        }
        oz_slice_tr_kernel<8><<<grid, 256, smem, st>>>(src, sz, sk, op.rows, op.K, op.rows_pad, op.kpitch,
                                                       op.nkb, op.expo, op.data, op.kblk);
        break;
      default:
        throw Error{DFJK_ERR_UNSUPPORTED, "slice count must be 6 or 8"};
    }
    DFJK_LAUNCHED();
    return;
  }
  const long long nt = (long long)op.batch * op.rows_pad * (op.kpitch / 8);
  const int row_fast = sk != 1;
  const unsigned grid = (unsigned)((nt + 255) / 256);
  switch (op.S) {
    case 6:
      oz_slice_kernel<6><<<grid, 256, 0, st>>>(src, sz, sr, sk, op.batch, op.rows, op.K, op.rows_pad,
                                               op.kpitch, op.nkb, op.expo, op.data, row_fast, op.kblk);
      break;
    case 8:
      oz_slice_kernel<8><<<grid, 256, 0, st>>>(src, sz, sr, sk, op.batch, op.rows, op.K, op.rows_pad,
                                               op.kpitch, op.nkb, op.expo, op.data, row_fast, op.kblk);
      break;
    default:
      throw Error{DFJK_ERR_UNSUPPORTED, "slice count must be 6 or 8"};
  }
  DFJK_LAUNCHED();
}

// ---- GEMM -----------------------------------------------------------------------

// Poll limit for the waits that wind a CTA down after an abort (copies and
// MMAs already issued must land before shared memory and TMEM are released);
// independent of the caller's timeout, which may be tiny in tests.
constexpr long long OZ_CLEANUP_POLLS = 1LL << 24;

// K per pipeline stage (one MMA deep; rows of 32 bytes).
constexpr int OZ_KS = 16;

// A stage: the S slices of the A tile, then a zero tile and the S slices of
// the B tile, so that B_{q}, B_{q+1} (q >= -1, B_{-1} the zero tile) form one
// 128-row K-major operand (oz_mma_step).
template <int S>
struct OzCfg {
  static constexpr int NST = (S <= 6) ? 5 : 4;
  static constexpr int A_TILE = OZ_BM * OZ_KS * 2;
  static constexpr int B_TILE = OZ_BN * OZ_KS * 2;
  static constexpr int ZERO = S * A_TILE;          // offset of the zero tile
  static constexpr int STAGE = S * A_TILE + (S + 1) * B_TILE;
  static constexpr int LOAD = S * (A_TILE + B_TILE);  // bytes TMA writes per stage
  static constexpr int SMEM = NST * STAGE + 1024 + 256;
  static_assert(S % 2 == 0 && S * OZ_BN <= 512, "TMEM holds S level accumulators of 64 columns");
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

// The MMAs of one K step of 16.  Level l (TMEM columns 64 l .. 64 l + 63)
// accumulates the slice products A_s B_t with s + t = l.  For each A slice s
// and each even level pair (r, r + 1) with r >= s - 1, one 128 x 128 MMA
// multiplies A_s by the stacked slices [B_{r-s}, B_{r-s+1}] (B_{-1} is the
// zero tile) into columns 64 r .. 64 r + 127: both levels at once, so A_s is
// read from shared memory once per pair of levels instead of once per level
// (12 MMAs for S = 6 and 20 for S = 8 where one per product would be 21 and
// 36 of half the width; the zero products cost 14% and 11% more tensor
// work).  Every MMA has the same shape and writes one of S / 2 disjoint
// column ranges, so the MMAs into one range are ordered by the tensor pipe.
// The first K step of a K-block starts each range (s = 0 comes first and
// covers every range).
template <int S>
__device__ __forceinline__ void oz_mma_step(uint32_t tbase, uint32_t sa, uint32_t &reg_init) {
  using Cfg = OzCfg<S>;
  constexpr uint32_t IDESC = tc::idesc_bf16(OZ_BM, 2 * OZ_BN);
  const uint32_t sz = sa + Cfg::ZERO;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const uint64_t ad = tc::sdesc_k_sw32(sa + s * Cfg::A_TILE);
#pragma unroll
    for (int r = s & ~1; r < S; r += 2) {
      const uint64_t bd = tc::sdesc_k_sw32(sz + (r - s + 1) * Cfg::B_TILE);
      tc::mma_bf16(tbase + r * OZ_BN, ad, bd, IDESC, (reg_init >> r) & 1u);
      reg_init |= 1u << r;
    }
  }
}

// Zeroes the zero tile of every stage (all threads of the CTA; a barrier
// follows before the first MMA).
template <int S>
__device__ __forceinline__ void oz_zero_tiles(uint8_t *smem) {
  using Cfg = OzCfg<S>;
  for (int i = threadIdx.x; i < Cfg::NST * (Cfg::B_TILE / 16); i += blockDim.x) {
    const int st = i / (Cfg::B_TILE / 16), o = i % (Cfg::B_TILE / 16);
    *reinterpret_cast<uint4 *>(smem + st * Cfg::STAGE + Cfg::ZERO + o * 16) = make_uint4(0, 0, 0, 0);
  }
  tc::fence_proxy_async_smem();
}

struct OzKernelArgs {
  OzGemmArgs g;
  const int *expoA, *expoB;
  int rows_padA, rows_padB, nkbA, nkbB;
  int kblkA, kblkB;  // K-blocked slice layouts (4-D tensor maps)
};

// 2^e for normal exponents; 0 below the normal range (row maxima that small
// do not occur for these operands except as exact zeros).
// TMA load of one slice tile: rows row0.. of slice plane `plane` at K offset kc.
__device__ __forceinline__ void oz_tma(void *dst, const CUtensorMap *map, uint64_t *bar, int kc, int row0,
                                       int plane, int kblk) {
  if (kblk) tc::tma_load_4d(dst, map, bar, kc & (OZ_KB - 1), row0, kc >> 10, plane);
  else tc::tma_load_3d(dst, map, bar, kc, row0, plane);
}

__device__ __forceinline__ double pow2(int e) {
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

// Recombination of the S level sums of one output (exact integers in FP32,
// |sum| < 2^23) into one int64: levels 0..TOP exactly, shifted by 6 bits per
// level; for S = 8 the last level is rounded to the unit of level 6, so that
// |T| < 2^60 (S <= 6: every level exact, |T| < 2^54).  The output value is
// T 2^(eA + eB - UNIT), one FP64 multiply-add per output and K block.
template <int S>
struct OzLev {
  static constexpr int TOP = (S <= 6) ? S - 1 : S - 2;
  static constexpr int UNIT = 12 + 6 * TOP;
};
template <int S>
__device__ __forceinline__ void oz_add_level(long long &T, int lev, float v) {
  const long long iv = (long long)__float2int_rn(v);
  if (lev <= OzLev<S>::TOP) T += iv << (6 * (OzLev<S>::TOP - lev));
  else T += (iv + (1LL << (6 * (lev - OzLev<S>::TOP) - 1))) >> (6 * (lev - OzLev<S>::TOP));
}

template <int S>
__global__ void __launch_bounds__(128, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const OzKernelArgs ka) {
  using Cfg = OzCfg<S>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + Cfg::NST * Cfg::STAGE);
  uint64_t *empty = full + Cfg::NST;
  uint64_t *accf = empty + Cfg::NST;
  uint32_t *tmem_holder = (uint32_t *)(accf + 1);

  const OzGemmArgs &g = ka.g;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * OZ_BM, n0 = blockIdx.y * OZ_BN, z = blockIdx.z;
  if (g.lower_only && n0 > m0 + OZ_BM - 1) return;
  int kb0 = 0, kb1 = (g.K + OZ_KB - 1) / OZ_KB, kend = g.K;
  if (g.kb_per_split > 0) {
    kb0 = z * g.kb_per_split;
    kb1 = min(kb1, kb0 + g.kb_per_split);
  }
  if (g.k_upto_n) {
    kend = min(kend, n0 + OZ_BN);
    kb1 = min(kb1, (kend + OZ_KB - 1) / OZ_KB);
  }
  const int zA = g.a_batched ? z : 0, zB = g.b_batched ? z : 0;

  if (warp == 0) tc::tmem_alloc(tmem_holder, 512);
  oz_zero_tiles<S>(smem);
  if (tid == 0) {
    for (int i = 0; i < Cfg::NST; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(accf, 1);
    tc::fence_mbar_init();
    tc::prefetch_tensormap(&tmA);
    tc::prefetch_tensormap(&tmB);
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_holder;

  double acc[OZ_BN];
#pragma unroll
  for (int j = 0; j < OZ_BN; ++j) acc[j] = 0.0;
  const int m = m0 + tid;
  uint32_t gstage = 0;  // stages consumed so far (thread 0)
  bool ok = true;
  int kbi = 0;
  for (int kb = kb0; kb < kb1; ++kb, ++kbi) {
    const int kstart = kb * OZ_KB;
    const int kstop = min(kend, kstart + OZ_KB);
    const int nst = (kstop - kstart + OZ_KS - 1) / OZ_KS;
    if (tid == 0) {
      uint32_t lev_init = 0;
      constexpr int dist = Cfg::NST - 1;
      int issued = 0, consumed = 0;
      for (int j = 0; j < nst + dist && ok; ++j) {
        if (j < nst) {
          const uint32_t gs = gstage + j, slot = gs % Cfg::NST;
          if (gs >= (uint32_t)Cfg::NST &&
              !tc::mbar_wait(&empty[slot], ((gs / Cfg::NST) - 1) & 1, g.timeout)) {
            ok = false;
            break;
          }
          uint8_t *stp = smem + slot * Cfg::STAGE;
          tc::mbar_expect_tx(&full[slot], Cfg::LOAD);
          const int kc = kstart + j * OZ_KS;
#pragma unroll
          for (int s = 0; s < S; ++s)
            oz_tma(stp + s * Cfg::A_TILE, &tmA, &full[slot], kc, m0, zA * S + s, ka.kblkA);
#pragma unroll
          for (int t = 0; t < S; ++t)
            oz_tma(stp + Cfg::ZERO + (t + 1) * Cfg::B_TILE, &tmB, &full[slot], kc, n0, zB * S + t, ka.kblkB);
          ++issued;
        }
        if (j >= dist) {
          const uint32_t gs = gstage + (j - dist), slot = gs % Cfg::NST;
          if (!tc::mbar_wait(&full[slot], (gs / Cfg::NST) & 1, g.timeout)) {
            ok = false;
            break;
          }
          ++consumed;
          tc::tc_fence_after();
          oz_mma_step<S>(tbase, tc::smem_u32(smem + slot * Cfg::STAGE), lev_init);
          tc::mma_commit(&empty[slot]);
        }
      }
      if (ok) {
        tc::mma_commit(accf);
        gstage += nst;
      } else {
        if (g.status) atomicOr(g.status, STATUS_TIMEOUT);
        // copies still in flight land, and issued MMAs finish, before the CTA leaves
        for (int c = consumed; c < issued; ++c) {
          const uint32_t gs = gstage + c, slot = gs % Cfg::NST;
          tc::mbar_wait(&full[slot], (gs / Cfg::NST) & 1, OZ_CLEANUP_POLLS);
        }
        if (consumed > 0) {
          tc::mma_commit(accf);
          tc::mbar_wait(accf, kbi & 1, OZ_CLEANUP_POLLS);
        }
      }
    }
    // every thread: wait for this K-block's MMAs (bounded)
    if (!tc::mbar_wait(accf, kbi & 1, g.timeout)) ok = false;
    ok = __syncthreads_and(ok);
    if (!ok) {
      if (tid == 0 && g.status) atomicOr(g.status, STATUS_TIMEOUT);
      break;
    }
    tc::tc_fence_after();
    const int eA = ka.expoA[((long long)zA * ka.rows_padA + m) * ka.nkbA + kb] - OzLev<S>::UNIT;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c = 0; c < OZ_BN / 16; ++c) {
      long long T[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) T[j] = 0;
#pragma unroll
      for (int lev = 0; lev < S; ++lev) {
        float v[16];
        tc::tmem_ld16(tbase + lane_base + lev * OZ_BN + c * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) oz_add_level<S>(T[j], lev, v[j]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + c * 16 + j;
        const int eB = __ldg(ka.expoB + ((long long)zB * ka.rows_padB + n) * ka.nkbB + kb);
        acc[c * 16 + j] = fma((double)T[j], pow2(eA + eB), acc[c * 16 + j]);
      }
    }
    tc::tc_fence_before();
    __syncthreads();
  }

  if (ok && m < g.M) {
    double *o = g.out + (long long)z * g.out_bs + (long long)m * g.ldo;
#pragma unroll
    for (int j = 0; j < OZ_BN; ++j)
      if (n0 + j < g.N) o[n0 + j] = acc[j];
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// ---- persistent warp-specialised GEMM -----------------------------------------------
//
// 64 + 32 NEPI threads: warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM
// owner), warps 2.. = epilogue (warp w reads TMEM lanes 32 (w % 4) .. +31 and
// one column group of 64 / (NEPI / 4) columns).  Tile order: n fastest, so
// tiles in flight at the same time share their A rows.
// Tiles are handed out dynamically: the producer takes the next tile index
// from a global counter and passes it to the MMA and epilogue warps through a
// small queue in shared memory, so the CTAs advance through the tile order
// together and the operands of the tiles in flight stay in L2 (a static
// round-robin lets CTAs drift apart when tiles differ in length).  Per
// K-block: the producer fills the stage ring, the MMA warp accumulates S
// levels in TMEM and commits `accf`; the epilogue drains into FP64 registers
// and releases TMEM through `acce` (32 NEPI arrivals).  The producer runs
// ahead into the next K-block / tile during the drain.  (Releasing TMEM
// before the FP64 part of the drain, so that the next K block's MMAs overlap
// it, measured slower: holding the level sums and the accumulators together
// spilled at this kernel's register cap.)
// 8 drain warps: 4 TMEM lane quarters x 2 column halves of 32.
constexpr int OZ_NEPI = 8;
__host__ __device__ constexpr int oz_ws_threads(int nepi) { return 64 + 32 * nepi; }
constexpr int OZ_QD = 4;  // depth of the tile queue

struct OzTiles {
  int ntm, ntn, nz, total;
};

__device__ __forceinline__ bool oz_tile(const OzGemmArgs &g, const OzTiles &T, int t, int &m0, int &n0, int &z,
                                        int &kb0, int &kb1, int &kend) {
  const int tn = t % T.ntn, tm = (t / T.ntn) % T.ntm;
  z = t / (T.ntn * T.ntm);
  m0 = tm * OZ_BM;
  n0 = tn * OZ_BN;
  if (g.lower_only && n0 > m0 + OZ_BM - 1) return false;
  kb0 = 0;
  kb1 = (g.K + OZ_KB - 1) / OZ_KB;
  kend = g.K;
  if (g.kb_per_split > 0) {
    kb0 = z * g.kb_per_split;
    kb1 = min(kb1, kb0 + g.kb_per_split);
  }
  if (g.k_upto_n) {
    kend = min(kend, n0 + OZ_BN);
    kb1 = min(kb1, (kend + OZ_KB - 1) / OZ_KB);
  }
  return kb0 < kb1;
}

template <int S, int NEPI>
__global__ void __launch_bounds__(oz_ws_threads(NEPI), 1)
    oz_gemm_ws_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const OzKernelArgs ka, const OzTiles T) {
  using Cfg = OzCfg<S>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + Cfg::NST * Cfg::STAGE);
  uint64_t *empty = full + Cfg::NST;
  uint64_t *accf = empty + Cfg::NST;
  uint64_t *acce = accf + 1;
  uint64_t *fin = acce + 1;
  uint64_t *tqf = fin + 1;     // tile queue: slot filled (producer arrives)
  uint64_t *tqe = tqf + OZ_QD; // slot read (MMA warp + 8 epilogue warps arrive)
  uint32_t *tmem_holder = (uint32_t *)(tqe + OZ_QD);
  volatile int *abort_flag = (volatile int *)(tmem_holder + 1);
  volatile int *tq = (volatile int *)(tmem_holder + 2);  // OZ_QD tile indices (-1: no more)

  const OzGemmArgs &g = ka.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int OZ_WS_THREADS = oz_ws_threads(NEPI);
  if (warp == 1) tc::tmem_alloc(tmem_holder, 512);
  oz_zero_tiles<S>(smem);
  if (tid == 0) {
    for (int i = 0; i < Cfg::NST; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < OZ_QD; ++i) {
      tc::mbar_init(&tqf[i], 1);
      tc::mbar_init(&tqe[i], 1 + NEPI);
    }
    tc::mbar_init(accf, 1);
    tc::mbar_init(acce, OZ_WS_THREADS - 64);
    tc::mbar_init(fin, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tensormap(&tmA);
    tc::prefetch_tensormap(&tmB);
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_holder;
  const long long lim = g.timeout;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      uint32_t gs = 0, qi = 0;
      bool ok = true;
      while (ok) {
        int t, m0 = 0, n0 = 0, z = 0, kb0 = 0, kb1 = 0, kend = 0;
        do {
          t = atomicAdd(g.tile_ctr, 1);
        } while (t < T.total && !oz_tile(g, T, t, m0, n0, z, kb0, kb1, kend));
        const uint32_t qs = qi % OZ_QD;
        if (qi >= (uint32_t)OZ_QD && !tc::mbar_wait(&tqe[qs], ((qi / OZ_QD) - 1) & 1, lim)) {
          ok = false;
          break;
        }
        tq[qs] = t < T.total ? t : -1;
        tc::mbar_arrive(&tqf[qs]);
        ++qi;
        if (t >= T.total) break;
        const int zA = g.a_batched ? z : 0, zB = g.b_batched ? z : 0;
        for (int kb = kb0; kb < kb1 && ok; ++kb) {
          const int kstart = kb * OZ_KB, kstop = min(kend, kstart + OZ_KB);
          for (int kc = kstart; kc < kstop; kc += OZ_KS, ++gs) {
            const uint32_t slot = gs % Cfg::NST;
            if (gs >= (uint32_t)Cfg::NST && !tc::mbar_wait(&empty[slot], ((gs / Cfg::NST) - 1) & 1, lim)) {
              ok = false;
              break;
            }
            if (*abort_flag) {
              ok = false;
              break;
            }
            uint8_t *stp = smem + slot * Cfg::STAGE;
            tc::mbar_expect_tx(&full[slot], Cfg::LOAD);
#pragma unroll
            for (int s = 0; s < S; ++s)
              oz_tma(stp + s * Cfg::A_TILE, &tmA, &full[slot], kc, m0, zA * S + s, ka.kblkA);
#pragma unroll
            for (int q = 0; q < S; ++q)
              oz_tma(stp + Cfg::ZERO + (q + 1) * Cfg::B_TILE, &tmB, &full[slot], kc, n0, zB * S + q, ka.kblkB);
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (g.status) atomicOr(g.status, STATUS_TIMEOUT);
      }
      // copies in flight (the last NST stages issued) land before the CTA leaves
      for (uint32_t k = (gs > (uint32_t)Cfg::NST ? gs - Cfg::NST : 0); k < gs; ++k)
        tc::mbar_wait(&full[k % Cfg::NST], (k / Cfg::NST) & 1, OZ_CLEANUP_POLLS);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      uint32_t gs = 0, kbi = 0, qi = 0;
      bool ok = true;
      while (ok) {
        const uint32_t qs = qi % OZ_QD;
        if (!tc::mbar_wait(&tqf[qs], (qi / OZ_QD) & 1, lim) || *abort_flag) {
          ok = false;
          break;
        }
        const int t = tq[qs];
        tc::mbar_arrive(&tqe[qs]);
        ++qi;
        if (t < 0) break;
        int m0, n0, z, kb0, kb1, kend;
        oz_tile(g, T, t, m0, n0, z, kb0, kb1, kend);
        for (int kb = kb0; kb < kb1 && ok; ++kb, ++kbi) {
          if (kbi > 0 && !tc::mbar_wait(acce, (kbi - 1) & 1, lim)) {  // TMEM drained
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const int kstart = kb * OZ_KB, kstop = min(kend, kstart + OZ_KB);
          uint32_t lev_init = 0;
          for (int kc = kstart; kc < kstop; kc += OZ_KS, ++gs) {
            const uint32_t slot = gs % Cfg::NST;
            if (!tc::mbar_wait(&full[slot], (gs / Cfg::NST) & 1, lim) || *abort_flag) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            oz_mma_step<S>(tbase, tc::smem_u32(smem + slot * Cfg::STAGE), lev_init);
            tc::mma_commit(&empty[slot]);
          }
          if (ok) tc::mma_commit(accf);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (g.status) atomicOr(g.status, STATUS_TIMEOUT);
      }
      // every MMA issued has finished before TMEM is released
      tc::mma_commit(fin);
      tc::mbar_wait(fin, 0, OZ_CLEANUP_POLLS);
    }
  } else {  // ---- epilogue, 16 warps: TMEM lane group (warp % 4), column quarter
    const int lgrp = warp & 3;
    const int half = (warp - 2) >> 2;  // column group: columns NH half .. NH half + NH - 1
    const int row = lgrp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(lgrp * 32) << 16;
    constexpr int NH = OZ_BN / (NEPI / 4);
    uint32_t kbi = 0, qi = 0;
    bool ok = true;
    while (ok) {
      const uint32_t qs = qi % OZ_QD;
      const bool got = tc::mbar_wait(&tqf[qs], (qi / OZ_QD) & 1, lim);
      if (!__all_sync(0xffffffffu, got && !*abort_flag)) {
        ok = false;
        break;
      }
      const int t = tq[qs];
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tqe[qs]);
      ++qi;
      if (t < 0) break;
      int m0, n0, z, kb0, kb1, kend;
      oz_tile(g, T, t, m0, n0, z, kb0, kb1, kend);
      const int zA = g.a_batched ? z : 0, zB = g.b_batched ? z : 0;
      const int m = m0 + row;
      const int nh = n0 + half * NH;
      double acc[NH];
#pragma unroll
      for (int j = 0; j < NH; ++j) acc[j] = 0.0;
      for (int kb = kb0; kb < kb1; ++kb, ++kbi) {
        // warp-uniform decision: tcgen05.ld below needs the whole warp
        const bool waited = tc::mbar_wait(accf, kbi & 1, lim);
        if (!__all_sync(0xffffffffu, waited && !*abort_flag)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const int eA = ka.expoA[((long long)zA * ka.rows_padA + m) * ka.nkbA + kb] - OzLev<S>::UNIT;
        // this warp's 32 column exponents, one per lane, broadcast by shuffles
        const int eBl = __ldg(ka.expoB + ((long long)zB * ka.rows_padB + nh + lane) * ka.nkbB + kb);
#pragma unroll
        for (int c = 0; c < NH / 16; ++c) {
          long long Tv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) Tv[j] = 0;
#pragma unroll
          for (int lev = 0; lev < S; ++lev) {
            float v[16];
            tc::tmem_ld16(tbase + lane_base + lev * OZ_BN + half * NH + c * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) oz_add_level<S>(Tv[j], lev, v[j]);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int eB = __shfl_sync(0xffffffffu, eBl, c * 16 + j);
            acc[c * 16 + j] = fma((double)Tv[j], pow2(eA + eB), acc[c * 16 + j]);
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(acce);
      }
      if (!ok) break;
      if (g.mode == 2) {
        // split z of this tile adds onto splits 0..z-1 in order: wait until the
        // same drain warp of split z-1 has stored (bounded), then read-add-store
        int *seq = g.tile_seq + ((long long)(m0 / OZ_BM) * T.ntn + n0 / OZ_BN) * NEPI + (warp - 2);
        bool ready = true;
        if (lane == 0 && z > 0) {
          long long i = 0;
          while (*(volatile int *)seq != z) {
            if (++i > lim) {
              ready = false;
              break;
            }
            __nanosleep(64);
          }
        }
        if (!__shfl_sync(0xffffffffu, ready ? 1 : 0, 0)) {
          ok = false;
          break;
        }
        __threadfence();
        if (m < g.M) {
          double *o = g.out + (long long)m * g.ldo + nh;
#pragma unroll
          for (int j = 0; j < NH; ++j)
            if (nh + j < g.N) o[j] = (z == 0 && !g.accumulate) ? acc[j] : __ldcg(o + j) + acc[j];  // L2, not a stale L1 line
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) *(volatile int *)seq = z + 1;
      } else if (m < g.M) {
        const bool full = nh + NH <= g.N;
        double *o = g.out + (long long)z * g.out_bs + (long long)m * g.ldo + nh;
        if (full && ((uintptr_t)o & 15) == 0) {
#pragma unroll
          for (int j = 0; j < NH; j += 2) *reinterpret_cast<double2 *>(o + j) = make_double2(acc[j], acc[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < NH; ++j)
            if (nh + j < g.N) o[j] = acc[j];
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (g.status) atomicOr(g.status, STATUS_TIMEOUT);
    }
  }
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

// ---- host ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    DFJK_CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess)
      throw Error{DFJK_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

static CUtensorMap make_map(const SlicedOp &op, int box_rows) {
  CUtensorMap map;
  CUresult r;
  if (!op.kblk) {  // (k, row, batch x slice)
    cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows_pad, (cuuint64_t)op.batch * op.S};
    cuuint64_t strides[2] = {(cuuint64_t)op.kpitch * 2, (cuuint64_t)op.rows_pad * op.kpitch * 2};
    cuuint32_t box[3] = {OZ_KS, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.data, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {  // (k within block, row, K block, batch x slice); padding of the last block is zero
    cuuint64_t dims[4] = {(cuuint64_t)OZ_KB, (cuuint64_t)op.rows_pad, (cuuint64_t)op.nkb,
                          (cuuint64_t)op.batch * op.S};
    cuuint64_t strides[3] = {(cuuint64_t)OZ_KB * 2, (cuuint64_t)op.rows_pad * OZ_KB * 2,
                             (cuuint64_t)op.nkb * op.rows_pad * OZ_KB * 2};
    cuuint32_t box[4] = {OZ_KS, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, op.data, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) throw Error{DFJK_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
  return map;
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    DFJK_CUDA_CHECK(cudaGetDevice(&dev));
    DFJK_CUDA_CHECK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

// Persistent warp-specialised launch (the default).
template <int S, int NEPI>
static void launch_oz_ws_n(const SlicedOp &A, const SlicedOp &B, const OzGemmArgs &g, cudaStream_t st) {
  PhaseScope ph(g.phase, st);
  constexpr int SMEM = OzCfg<S>::SMEM;
  static bool attr_set = false;
  if (!attr_set) {
    DFJK_CUDA_CHECK(
        cudaFuncSetAttribute(oz_gemm_ws_kernel<S, NEPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    attr_set = true;
  }
  const CUtensorMap ma = make_map(A, OZ_BM), mb = make_map(B, OZ_BN);
  OzKernelArgs ka{g, A.expo, B.expo, A.rows_pad, B.rows_pad, A.nkb, B.nkb, A.kblk, B.kblk};
  OzTiles T;
  T.ntm = (g.M + OZ_BM - 1) / OZ_BM;
  T.ntn = (g.N + OZ_BN - 1) / OZ_BN;
  T.nz = g.nz;
  const long long total = (long long)T.ntm * T.ntn * T.nz;
  if (total > 2147483647LL) throw Error{DFJK_ERR_ARG, "oz_gemm: too many tiles"};
  T.total = (int)total;
  const int grid = (int)std::min<long long>(total, num_sms());
  if (!g.tile_ctr) throw Error{DFJK_ERR_ARG, "oz_gemm: tile counter"};
  DFJK_CUDA_CHECK(cudaMemsetAsync(g.tile_ctr, 0, sizeof(int), st));
  if (g.mode == 2) {
    if (!g.tile_seq || g.kb_per_split <= 0 || g.a_batched || g.b_batched)
      throw Error{DFJK_ERR_ARG, "oz_gemm: ordered split-K arguments"};
    DFJK_CUDA_CHECK(cudaMemsetAsync(g.tile_seq, 0, oz_tile_seq_count(g.M, g.N) * sizeof(int), st));
  }
  oz_gemm_ws_kernel<S, NEPI><<<grid, oz_ws_threads(NEPI), SMEM, st>>>(ma, mb, ka, T);
  DFJK_LAUNCHED();
}

template <int S>
static void launch_oz_ws(const SlicedOp &A, const SlicedOp &B, const OzGemmArgs &g, cudaStream_t st) {
  launch_oz_ws_n<S, OZ_NEPI>(A, B, g, st);
}

template <int S>
static void launch_oz(const SlicedOp &A, const SlicedOp &B, const OzGemmArgs &g, cudaStream_t st) {
  PhaseScope ph(g.phase, st);
  static bool attr_set = false;
  if (!attr_set) {
    DFJK_CUDA_CHECK(cudaFuncSetAttribute(oz_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<S>::SMEM));
    attr_set = true;
  }
  const CUtensorMap ma = make_map(A, OZ_BM), mb = make_map(B, OZ_BN);
  OzKernelArgs ka{g, A.expo, B.expo, A.rows_pad, B.rows_pad, A.nkb, B.nkb, A.kblk, B.kblk};
  dim3 grid((unsigned)((g.M + OZ_BM - 1) / OZ_BM), (unsigned)((g.N + OZ_BN - 1) / OZ_BN), (unsigned)g.nz);
  oz_gemm_kernel<S><<<grid, 128, OzCfg<S>::SMEM, st>>>(ma, mb, ka);
  DFJK_LAUNCHED();
}

bool oz_simple_mode() {
  static const bool simple = [] {
    const char *e = std::getenv("DFJK_OZ_SIMPLE");
    return e && e[0] == '1';
  }();
  return simple;
}

size_t oz_tile_seq_count(int M, int N) {
  return (size_t)((M + OZ_BM - 1) / OZ_BM) * ((N + OZ_BN - 1) / OZ_BN) * OZ_NEPI;
}

void oz_gemm(const SlicedOp &A, const SlicedOp &B, const OzGemmArgs &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.nz <= 0) return;
  if (A.S != B.S) throw Error{DFJK_ERR_ARG, "oz_gemm: slice counts differ"};
  if (A.K != B.K || A.K < g.K) throw Error{DFJK_ERR_ARG, "oz_gemm: K mismatch"};
  if (A.rows_pad % OZ_BM || B.rows_pad % OZ_BN) throw Error{DFJK_ERR_ARG, "oz_gemm: row padding"};
  if ((long long)((g.M + OZ_BM - 1) / OZ_BM) * OZ_BM > A.rows_pad ||
      (long long)((g.N + OZ_BN - 1) / OZ_BN) * OZ_BN > B.rows_pad)
    throw Error{DFJK_ERR_ARG, "oz_gemm: tiles exceed the padded operands"};
  if (g.a_batched && g.nz > A.batch) throw Error{DFJK_ERR_ARG, "oz_gemm: A batch"};
  if (g.b_batched && g.nz > B.batch) throw Error{DFJK_ERR_ARG, "oz_gemm: B batch"};
  if (g.mode != 0 && g.mode != 2) throw Error{DFJK_ERR_ARG, "oz_gemm: mode"};
  if (g.nz > 65535 || (g.M + OZ_BM - 1) / OZ_BM > 2147483647) throw Error{DFJK_ERR_ARG, "oz_gemm: grid"};
  const bool simple = oz_simple_mode();
  if (simple && g.mode == 2) throw Error{DFJK_ERR_UNSUPPORTED, "oz_gemm: mode 2 needs the persistent kernel"};
  switch (A.S) {
    case 6: simple ? launch_oz<6>(A, B, g, st) : launch_oz_ws<6>(A, B, g, st); break;
    case 8: simple ? launch_oz<8>(A, B, g, st) : launch_oz_ws<8>(A, B, g, st); break;
    default: throw Error{DFJK_ERR_UNSUPPORTED, "slice count must be 6 or 8"};
  }
}

}  // namespace dfjk

// Debug entry point for tests: C[z][m][n] = sum_k A[z][m][k] B[n][k] through
// slicing + the tensor-core GEMM (A, B, C device FP64 row-major).
extern "C" int dfjk_debug_sliced_gemm(int32_t batch, int32_t M, int32_t N, int32_t K, int32_t S,
                                      const double *A, const double *B, double *C, int32_t *status,
                                      void *stream) {
  using namespace dfjk;
  SlicedOp a, b;
  int *ctr = nullptr;
  try {
    if (batch < 1 || M < 1 || N < 1 || K < 1 || !A || !B || !C) throw Error{DFJK_ERR_ARG, "sliced gemm arguments"};
    cudaStream_t st = (cudaStream_t)stream;
    ctr = (int *)pool_alloc(sizeof(int));
    oz_alloc(a, batch, S, M, K, OZ_BM);
    oz_alloc(b, 1, S, N, K, OZ_BN);
    oz_slice_f64(A, (long long)M * K, K, 1, a, st);
    oz_slice_f64(B, 0, K, 1, b, st);
    OzGemmArgs g;
    g.M = M; g.N = N; g.K = K; g.nz = batch; g.a_batched = 1;
    g.mode = 0; g.out = C; g.ldo = N; g.out_bs = (long long)M * N;
    g.status = (int *)status;
    g.tile_ctr = ctr;
    oz_gemm(a, b, g, st);
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    oz_free(a);
    oz_free(b);
    pool_free(ctr, sizeof(int));
    return DFJK_OK;
  } catch (const Error &e) {
    cudaStreamSynchronize((cudaStream_t)stream);
    oz_free(a);
    oz_free(b);
    if (ctr) pool_free(ctr, sizeof(int));
    set_error(e.msg);
    return e.code;
  }
}
