// McMurchie-Davidson kernel templates shared by the integral translation units.
// The scheme and its equations are described in integrals.cu.
#pragma once

#include <cstdlib>

#include "boys.cuh"
#include "common.cuh"
#include "integrals.cuh"

namespace dfjk {


// ---- Hermite index helpers ---------------------------------------------------

__host__ __device__ constexpr int ntuv(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
// Dense index of (t,u,v): levels n = t+u+v, then descending t, then descending u.
__host__ __device__ constexpr int tuv_idx(int t, int u, int v) {
  return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// Number of (component pair, t, u, v) terms of a shell-pair class.
__host__ __device__ constexpr int nterms(int LA, int LB) {
  int n = 0;
  for (int ca = 0; ca < ncart(LA); ++ca)
    for (int cb = 0; cb < ncart(LB); ++cb)
      n += (cart_x(LA, ca) + cart_x(LB, cb) + 1) * (cart_y(LA, ca) + cart_y(LB, cb) + 1) *
           (cart_z(LA, ca) + cart_z(LB, cb) + 1);
  return n;
}


// R^0_{tuv} for t+u+v <= L (Real = double, or float for the FP32 pairs).
template <int L, typename Real = double>
__device__ __forceinline__ void hermite_R(const Real *F, Real a, Real X, Real Y, Real Z, Real *R) {
  Real pw[L + 1];
  pw[0] = Real(1);
#pragma unroll
  for (int n = 1; n <= L; ++n) pw[n] = pw[n - 1] * (Real(-2) * a);
  Real cur[ntuv(L)];
  cur[0] = pw[L] * F[L];
#pragma unroll
  for (int n = L - 1; n >= 0; --n) {
    Real nxt[ntuv(L)];
    nxt[0] = pw[n] * F[n];
#pragma unroll
    for (int N = 1; N <= L - n; ++N)
#pragma unroll
      for (int t = N; t >= 0; --t)
#pragma unroll
        for (int u = N - t; u >= 0; --u) {
          const int v = N - t - u;
          Real r;
          if (t > 0) {
            r = X * cur[tuv_idx(t - 1, u, v)];
            if (t > 1) r = fma(Real(t - 1), cur[tuv_idx(t - 2, u, v)], r);
          } else if (u > 0) {
            r = Y * cur[tuv_idx(t, u - 1, v)];
            if (u > 1) r = fma(Real(u - 1), cur[tuv_idx(t, u - 2, v)], r);
          } else {
            r = Z * cur[tuv_idx(t, u, v - 1)];
            if (v > 1) r = fma(Real(v - 1), cur[tuv_idx(t, u, v - 2)], r);
          }
          nxt[tuv_idx(t, u, v)] = r;
        }
#pragma unroll
    for (int k = 0; k < ntuv(L - n); ++k) cur[k] = nxt[k];
  }
#pragma unroll
  for (int k = 0; k < ntuv(L); ++k) R[k] = cur[k];
}

// Same recursion with a runtime order (L <= 8), loops not unrolled: used by
// the Schwarz diagonal, where compile time matters more than speed.
template <typename Real>
static __device__ __noinline__ void hermite_R_rt(int L, const Real *F, Real a, Real X, Real Y, Real Z, Real *R) {
  Real cur[ntuv(8)], nxt[ntuv(8)];
  Real pw = 1;
  for (int n = 0; n < L; ++n) pw *= Real(-2) * a;
  cur[0] = pw * F[L];
#pragma unroll 1
  for (int n = L - 1; n >= 0; --n) {
    pw = 1;
    for (int k = 0; k < n; ++k) pw *= Real(-2) * a;
    nxt[0] = pw * F[n];
#pragma unroll 1
    for (int N = 1; N <= L - n; ++N)
#pragma unroll 1
      for (int t = N; t >= 0; --t)
#pragma unroll 1
        for (int u = N - t; u >= 0; --u) {
          const int v = N - t - u;
          Real r;
          if (t > 0) {
            r = X * cur[tuv_idx(t - 1, u, v)];
            if (t > 1) r = fma(Real(t - 1), cur[tuv_idx(t - 2, u, v)], r);
          } else if (u > 0) {
            r = Y * cur[tuv_idx(t, u - 1, v)];
            if (u > 1) r = fma(Real(u - 1), cur[tuv_idx(t, u - 2, v)], r);
          } else {
            r = Z * cur[tuv_idx(t, u, v - 1)];
            if (v > 1) r = fma(Real(v - 1), cur[tuv_idx(t, u, v - 2)], r);
          }
          nxt[tuv_idx(t, u, v)] = r;
        }
    for (int k = 0; k < ntuv(L - n); ++k) cur[k] = nxt[k];
  }
  for (int k = 0; k < ntuv(L); ++k) R[k] = cur[k];
}

// E^{ij}_t for one direction, i <= LA, j <= LB (t <= i+j), with E^{00}_0 = 1.
template <int LA, int LB>
__device__ __forceinline__ void hermite_E(double inv2p, double XPA, double XPB,
                                          double E[LA + 1][LB + 1][LA + LB + 1]) {
#pragma unroll
  for (int i = 0; i <= LA; ++i)
#pragma unroll
    for (int j = 0; j <= LB; ++j)
#pragma unroll
      for (int t = 0; t <= LA + LB; ++t) E[i][j][t] = 0.0;
  E[0][0][0] = 1.0;
#pragma unroll
  for (int i = 0; i <= LA; ++i)
#pragma unroll
    for (int j = 0; j <= LB; ++j) {
      if (i == 0 && j == 0) continue;
      if (i > 0) {
#pragma unroll
        for (int t = 0; t <= i + j; ++t) {
          double e = XPA * E[i - 1][j][t];
          if (t > 0) e = fma(inv2p, E[i - 1][j][t - 1], e);
          if (t + 1 <= i - 1 + j) e = fma((double)(t + 1), E[i - 1][j][t + 1], e);
          E[i][j][t] = e;
        }
      } else {
#pragma unroll
        for (int t = 0; t <= j; ++t) {
          double e = XPB * E[0][j - 1][t];
          if (t > 0) e = fma(inv2p, E[0][j - 1][t - 1], e);
          if (t + 1 <= j - 1) e = fma((double)(t + 1), E[0][j - 1][t + 1], e);
          E[0][j][t] = e;
        }
      }
    }
}

// ---- pair kernel: primitive-pair records and Schwarz diagonal ----------------

// One thread per shell pair of class (LA, LB).  Record of a primitive pair:
//   [0] p  [1..3] P  [4] c_a c_b K_ab 2 pi^(5/2)/p  [5..] E^x E^y E^z per term.
// q[pair] = sqrt(max over components of (ab|ab)), the Schwarz factor.
template <int LA, int LB>
__global__ void __launch_bounds__(128) pair_kernel(PairClassArgs args, OrbArgs orb,
                                                   const double *__restrict__ boys_tab) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= args.npair) return;
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB);
  const int sa = args.shell_a[ip], sb = args.shell_b[ip];
  const double Ax = orb.center[3 * sa], Ay = orb.center[3 * sa + 1], Az = orb.center[3 * sa + 2];
  const double Bx = orb.center[3 * sb], By = orb.center[3 * sb + 1], Bz = orb.center[3 * sb + 2];
  const double ABx = Ax - Bx, ABy = Ay - By, ABz = Az - Bz;
  const double AB2 = ABx * ABx + ABy * ABy + ABz * ABz;
  double *rec0 = args.rec + args.rec_off[ip];
  const int pa0 = orb.prim_off[sa], na = orb.nprim[sa];
  const int pb0 = orb.prim_off[sb], nb = orb.nprim[sb];
  int npp = 0;
  for (int ka = 0; ka < na; ++ka)
    for (int kb = 0; kb < nb; ++kb, ++npp) {
      const double a = orb.exps[pa0 + ka], b = orb.exps[pb0 + kb];
      const double p = a + b, ip_ = 1.0 / p;
      const double Px = (a * Ax + b * Bx) * ip_, Py = (a * Ay + b * By) * ip_,
                   Pz = (a * Az + b * Bz) * ip_;
      double *r = rec0 + (long long)npp * REC;
      r[0] = p;
      r[1] = Px;
      r[2] = Py;
      r[3] = Pz;
      r[4] = orb.coefs[pa0 + ka] * orb.coefs[pb0 + kb] * exp(-a * b * ip_ * AB2) *
             (2.0 * 17.493418327624862846 * ip_);  // 2 pi^(5/2) / p
      double Ex[LA + 1][LB + 1][LA + LB + 1], Ey[LA + 1][LB + 1][LA + LB + 1],
          Ez[LA + 1][LB + 1][LA + LB + 1];
      const double inv2p = 0.5 * ip_;
      hermite_E<LA, LB>(inv2p, Px - Ax, Px - Bx, Ex);
      hermite_E<LA, LB>(inv2p, Py - Ay, Py - By, Ey);
      hermite_E<LA, LB>(inv2p, Pz - Az, Pz - Bz, Ez);
      int k = 0;
#pragma unroll
      for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
        for (int cb = 0; cb < NCB; ++cb) {
          const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
          const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
#pragma unroll
          for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
            for (int u = 0; u <= ay + by; ++u)
#pragma unroll
              for (int v = 0; v <= az + bz; ++v) r[REC_HDR + k++] = Ex[ax][bx][t] * Ey[ay][by][u] * Ez[az][bz][v];
        }
    }

}


// Schwarz factor q = sqrt(max over components of (ab|ab)) for every shell pair
// of class (LA, LB): one block per pair, one thread per primitive quadruple
// (kl, k'l') of the pair's records, then a block reduction.  Runtime loops:
// this is a small share of the work and unrolling it costs minutes of compile.
template <int LA, int LB, typename Real>
__global__ void __launch_bounds__(64) schwarz_kernel(PairClassArgs args, const Real *__restrict__ boys_tab) {
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB);
  constexpr int L4 = 2 * (LA + LB);
  __shared__ Real red[64][NCA * NCB + 1];
  const int ip = blockIdx.x;
  const double *rec0 = args.rec + args.rec_off[ip];
  const int npp = args.npp_of[ip];
  Real diag[NCA * NCB];
  for (int c = 0; c < NCA * NCB; ++c) diag[c] = 0;
#pragma unroll 1
  for (int q = threadIdx.x; q < npp * npp; q += blockDim.x) {
    const double *ri = rec0 + (long long)(q / npp) * REC;
    const double *rj = rec0 + (long long)(q % npp) * REC;
    const Real p = (Real)ri[0], qq = (Real)rj[0];
    const Real s = Real(1) / sqrt(p + qq);
    const Real al = p * qq * s * s;
    // centre differences in FP64 before rounding
    const Real X = (Real)(ri[1] - rj[1]), Y = (Real)(ri[2] - rj[2]), Z = (Real)(ri[3] - rj[3]);
    Real F[L4 + 1];
    boys_eval<L4>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
    Real R[ntuv(8)];
    hermite_R_rt<Real>(L4, F, al, X, Y, Z, R);
    // ri[4] rj[4] = c c K c c K (2 pi^2.5)^2 / (p q); wanted 2 pi^2.5 / (p q sqrt(p+q))
    const Real fac = (Real)(ri[4] * rj[4] * (1.0 / (2.0 * 17.493418327624862846))) * s;
    int k = 0;
#pragma unroll 1
    for (int ca = 0; ca < NCA; ++ca)
#pragma unroll 1
      for (int cb = 0; cb < NCB; ++cb) {
        const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
        const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
        const int k0 = k;
        Real sum = 0;
#pragma unroll 1
        for (int t = 0; t <= ax + bx; ++t)
#pragma unroll 1
          for (int u = 0; u <= ay + by; ++u)
#pragma unroll 1
            for (int v = 0; v <= az + bz; ++v) {
              Real inner = 0;
              int k2 = k0;
#pragma unroll 1
              for (int t2 = 0; t2 <= ax + bx; ++t2)
#pragma unroll 1
                for (int u2 = 0; u2 <= ay + by; ++u2)
#pragma unroll 1
                  for (int v2 = 0; v2 <= az + bz; ++v2) {
                    const Real e = (Real)rj[REC_HDR + k2];
                    const Real e2 = ((t2 + u2 + v2) & 1) ? -e : e;
                    inner = fma(e2, R[tuv_idx(t + t2, u + u2, v + v2)], inner);
                    ++k2;
                  }
              sum = fma((Real)ri[REC_HDR + k], inner, sum);
              ++k;
            }
        diag[ca * NCB + cb] = fma(fac, sum, diag[ca * NCB + cb]);
      }
  }
  for (int c = 0; c < NCA * NCB; ++c) red[threadIdx.x][c] = diag[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double qmax = 0.0;
    for (int ca = 0; ca < NCA; ++ca)
      for (int cb = 0; cb < NCB; ++cb) {
        Real d = 0;
        for (int t = 0; t < 64; ++t) d += red[t][ca * NCB + cb];
        const double f = comp_factor(LA, ca) * comp_factor(LB, cb);
        qmax = fmax(qmax, (double)d * f * f);
      }
    args.q[ip] = sqrt(fmax(qmax, 0.0));
  }
}

// ---- 3-centre kernel ---------------------------------------------------------

// Block: one shell pair of class (LA, LB) (blockIdx.x indexes the kept-pair
// list), 128 aux shells of class LC (blockIdx.y).  Thread: one aux shell;
// loops over the pair's primitive pairs (records staged in shared memory) and
// the aux primitives, accumulating the ncart(LA) ncart(LB) ncart(LC) block,
// then writes T[col - col_begin][P] (P contiguous).
template <int LA, int LB, int LC>
__global__ void __launch_bounds__(128) eri3c_kernel(Eri3cArgs args, AuxArgs aux,
                                                    const double *__restrict__ boys_tab) {
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB), NCC = ncart(LC);
  constexpr int LAB = LA + LB, L = LA + LB + LC;
  __shared__ double srec[REC];
  const int pair = args.pairs[blockIdx.x];
  const int as = blockIdx.y * blockDim.x + threadIdx.x;
  const bool active = as < args.naux_shells;
  const int sc = active ? args.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  double acc[NCA * NCB * NCC];
#pragma unroll
  for (int i = 0; i < NCA * NCB * NCC; ++i) acc[i] = 0.0;
  const double *rec0 = args.rec + args.rec_off[pair];
  const int npp = args.npp[pair];
  for (int ipp = 0; ipp < npp; ++ipp) {
    __syncthreads();
    for (int i = threadIdx.x; i < REC; i += blockDim.x) srec[i] = rec0[(long long)ipp * REC + i];
    __syncthreads();
    for (int kc = 0; kc < nc; ++kc) {
      const double g = aux.exps[pc0 + kc];
      const double g1 = aux.g1[pc0 + kc];  // 1/(2g)
      const double p = srec[0];
      const double X = srec[1] - Cx, Y = srec[2] - Cy, Z = srec[3] - Cz;
      const double s = rsqrt(p + g);
      const double al = p * g * (s * s);
      double F[L + 1];
      boys_eval<L>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
      double R[ntuv(L)];
      hermite_R<L>(F, al, X, Y, Z, R);
      const double pt = srec[4] * aux.cdiv[pc0 + kc] * s;  // c_c / g folded in cdiv
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc) {
        const int cx = cart_x(LC, cc), cy = cart_y(LC, cc), cz = cart_z(LC, cc);
        // W[tuv] for t+u+v <= LAB: aux Hermite expansion folded into shifts.
        double W[ntuv(LAB)];
        double scale = 1.0;
        if (LC == 0) {
#pragma unroll
          for (int i = 0; i < ntuv(LAB); ++i) W[i] = R[i];
        } else {
          const int two = (cx == 2) ? 0 : (cy == 2) ? 1 : (cz == 2) ? 2 : -1;
#pragma unroll
          for (int N = 0; N <= LAB; ++N)
#pragma unroll
            for (int t = N; t >= 0; --t)
#pragma unroll
              for (int u = N - t; u >= 0; --u) {
                const int v = N - t - u;
                if (two == 0)
                  W[tuv_idx(t, u, v)] = fma(g1, R[tuv_idx(t + 2, u, v)], R[tuv_idx(t, u, v)]);
                else if (two == 1)
                  W[tuv_idx(t, u, v)] = fma(g1, R[tuv_idx(t, u + 2, v)], R[tuv_idx(t, u, v)]);
                else if (two == 2)
                  W[tuv_idx(t, u, v)] = fma(g1, R[tuv_idx(t, u, v + 2)], R[tuv_idx(t, u, v)]);
                else
                  W[tuv_idx(t, u, v)] = R[tuv_idx(t + cx, u + cy, v + cz)];
              }
          if (two >= 0)
            scale = g1;
          else if (LC == 1)
            scale = -g1;
          else
            scale = g1 * g1;
        }
        const double ps = pt * scale;
        int k = 0;
#pragma unroll
        for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
          for (int cb = 0; cb < NCB; ++cb) {
            const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
            const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
            double sum = 0.0;
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
              for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                for (int v = 0; v <= az + bz; ++v) sum = fma(srec[REC_HDR + k++], W[tuv_idx(t, u, v)], sum);
            acc[(ca * NCB + cb) * NCC + cc] = fma(ps, sum, acc[(ca * NCB + cb) * NCC + cc]);
          }
      }
    }
  }
  if (!active) return;
  const long long col0 = args.pair_col[pair] - args.col_begin;
  const int P0 = aux.func_off[sc];
#pragma unroll
  for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb)
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc)
        args.T[(col0 + ca * NCB + cb) * args.ldT + P0 + cc] =
            acc[(ca * NCB + cb) * NCC + cc] *
            (comp_factor(LA, ca) * comp_factor(LB, cb) * comp_factor(LC, cc));
}

// FP32 variant for shell pairs whose Schwarz bound Q_ab max_P sqrt((P|P)) is
// below the FP32 threshold (the mixed-precision use of Schwarz estimates the
// paper names as future work in "Limitations and Future Development"): every
// integral of such a pair is below the bound, so FP32 rounding (relative
// ~1e-7 of the bound) stays far below the FP64 error of the large pairs after
// whitening.  Same loops as eri3c_kernel on the FP32 pipe (62x the FP64 rate
// here); the pair-to-aux-centre vector is formed in FP64 before rounding, so
// nearby centres keep their relative accuracy.
template <int LA, int LB, int LC>
__global__ void __launch_bounds__(128) eri3c32_kernel(Eri3cArgs args, AuxArgs aux,
                                                      const float *__restrict__ boys_tab) {
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB), NCC = ncart(LC);
  constexpr int LAB = LA + LB, L = LA + LB + LC;
  __shared__ double sP[3];
  __shared__ float srec[REC];
  const int pair = args.pairs[blockIdx.x];
  const int as = blockIdx.y * blockDim.x + threadIdx.x;
  const bool active = as < args.naux_shells;
  const int sc = active ? args.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  float acc[NCA * NCB * NCC];
#pragma unroll
  for (int i = 0; i < NCA * NCB * NCC; ++i) acc[i] = 0.0f;
  const double *rec0 = args.rec + args.rec_off[pair];
  const int npp = args.npp[pair];
  for (int ipp = 0; ipp < npp; ++ipp) {
    __syncthreads();
    for (int i = threadIdx.x; i < REC; i += blockDim.x) {
      const double v = rec0[(long long)ipp * REC + i];
      srec[i] = (float)v;
      if (i >= 1 && i <= 3) sP[i - 1] = v;
    }
    __syncthreads();
    const float X = (float)(sP[0] - Cx), Y = (float)(sP[1] - Cy), Z = (float)(sP[2] - Cz);
    for (int kc = 0; kc < nc; ++kc) {
      const float g = (float)aux.exps[pc0 + kc];
      const float g1 = (float)aux.g1[pc0 + kc];
      const float p = srec[0];
      const float s = rsqrtf(p + g);
      const float al = p * g * (s * s);
      float F[L + 1];
      boys_eval<L>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
      float R[ntuv(L)];
      hermite_R<L, float>(F, al, X, Y, Z, R);
      const float pt = srec[4] * (float)aux.cdiv[pc0 + kc] * s;
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc) {
        const int cx = cart_x(LC, cc), cy = cart_y(LC, cc), cz = cart_z(LC, cc);
        float W[ntuv(LAB)];
        float scale = 1.0f;
        if (LC == 0) {
#pragma unroll
          for (int i = 0; i < ntuv(LAB); ++i) W[i] = R[i];
        } else {
          const int two = (cx == 2) ? 0 : (cy == 2) ? 1 : (cz == 2) ? 2 : -1;
#pragma unroll
          for (int N = 0; N <= LAB; ++N)
#pragma unroll
            for (int t = N; t >= 0; --t)
#pragma unroll
              for (int u = N - t; u >= 0; --u) {
                const int v = N - t - u;
                if (two == 0)
                  W[tuv_idx(t, u, v)] = fmaf(g1, R[tuv_idx(t + 2, u, v)], R[tuv_idx(t, u, v)]);
                else if (two == 1)
                  W[tuv_idx(t, u, v)] = fmaf(g1, R[tuv_idx(t, u + 2, v)], R[tuv_idx(t, u, v)]);
                else if (two == 2)
                  W[tuv_idx(t, u, v)] = fmaf(g1, R[tuv_idx(t, u, v + 2)], R[tuv_idx(t, u, v)]);
                else
                  W[tuv_idx(t, u, v)] = R[tuv_idx(t + cx, u + cy, v + cz)];
              }
          if (two >= 0)
            scale = g1;
          else if (LC == 1)
            scale = -g1;
          else
            scale = g1 * g1;
        }
        const float ps = pt * scale;
        int k = 0;
#pragma unroll
        for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
          for (int cb = 0; cb < NCB; ++cb) {
            const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
            const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
            float sum = 0.0f;
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
              for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                for (int v = 0; v <= az + bz; ++v) sum = fmaf(srec[REC_HDR + k++], W[tuv_idx(t, u, v)], sum);
            acc[(ca * NCB + cb) * NCC + cc] = fmaf(ps, sum, acc[(ca * NCB + cb) * NCC + cc]);
          }
      }
    }
  }
  if (!active) return;
  const long long col0 = args.pair_col[pair] - args.col_begin;
  const int P0 = aux.func_off[sc];
#pragma unroll
  for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb)
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc)
        args.T[(col0 + ca * NCB + cb) * args.ldT + P0 + cc] =
            (double)acc[(ca * NCB + cb) * NCC + cc] *
            (comp_factor(LA, ca) * comp_factor(LB, cb) * comp_factor(LC, cc));
}

// ---- cooperative 3-centre kernel for aux shells with l >= 1 ------------------
//
// The one-thread-per-aux-shell kernels above keep every output of a shell
// triple in registers: 216 for (dd|d), plus R (84 terms at L = 6) and W, far
// beyond the 255 registers of a thread, so they spill to local memory and
// wait on it (ncu at 20 atoms: (dd|d) keeps the FP64 pipe 15 % busy).  Here
// the NCC = ncart(LC) threads of an aux shell (adjacent lanes of one warp)
// share its work: all of them evaluate the Boys function (free within the warp
// instruction), they build R^(n) level by level into shared memory, each
// computing every NCC-th entry, and then each thread forms W for its own aux
// component and contracts it with every orbital component pair: NCA NCB
// outputs (36 for dd) and ntuv(LAB) W terms (35) in registers.

// (t, u, v) of the k-th Hermite index in tuv_idx order, k < ntuv(8).
struct TuvTable {
  signed char t[ntuv(8)], u[ntuv(8)], v[ntuv(8)];
};
__host__ __device__ constexpr TuvTable make_tuv_table() {
  TuvTable T{};
  int k = 0;
  for (int n = 0; n <= 8; ++n)
    for (int t = n; t >= 0; --t)
      for (int u = n - t; u >= 0; --u) {
        T.t[k] = (signed char)t;
        T.u[k] = (signed char)u;
        T.v[k] = (signed char)(n - t - u);
        ++k;
      }
  return T;
}
// The recursion step of entry k >= 1 of R^(n) from R^(n+1), packed as
// idx1 | idx2 << 8 | dir << 16 | coef << 18: R_k = P_dir R'_idx1 + coef R'_idx2
// (dir 0, 1, 2 = the first of t, u, v that is > 0; coef = that index - 1, and
// idx2 = 0 when coef = 0).
struct RecTable {
  int e[ntuv(8)];
};
__host__ __device__ constexpr RecTable make_rec_table() {
  RecTable R{};
  const TuvTable T = make_tuv_table();
  for (int k = 1; k < ntuv(8); ++k) {
    const int t = T.t[k], u = T.u[k], v = T.v[k];
    int d = 0, i1 = 0, i2 = 0, c = 0;
    if (t > 0) {
      d = 0; i1 = tuv_idx(t - 1, u, v);
      if (t > 1) { c = t - 1; i2 = tuv_idx(t - 2, u, v); }
    } else if (u > 0) {
      d = 1; i1 = tuv_idx(t, u - 1, v);
      if (u > 1) { c = u - 1; i2 = tuv_idx(t, u - 2, v); }
    } else {
      d = 2; i1 = tuv_idx(t, u, v - 1);
      if (v > 1) { c = v - 1; i2 = tuv_idx(t, u, v - 2); }
    }
    R.e[k] = i1 | (i2 << 8) | (d << 16) | (c << 18);
  }
  return R;
}
__constant__ RecTable c_rec = make_rec_table();

__device__ __forceinline__ int tuv_idx_rt(int t, int u, int v) { return tuv_idx(t, u, v); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// Which kernel evaluates a class: the cooperative one where it measured
// faster (the classes whose one-thread kernel spills: (dp|p), (dp|d),
// (dd|p), (dd|d)); the one-thread kernel elsewhere, where every
// thread of a warp works on its own aux shell and the cooperative kernel's
// per-lane Boys evaluations would cost more than they save.  DFJK_ERI_COOP=0
// or 1 forces one kernel for every class with aux l >= 1.
inline bool eri3c_use_coop(int la, int lb, int lc, bool fp32) {
  static const int mode = [] {
    const char *e = std::getenv("DFJK_ERI_COOP");
    return e ? (e[0] == '0' ? 0 : (e[0] == '1' ? 1 : 2)) : 2;
  }();
  if (lc == 0 || mode == 0) return false;
  if (mode == 1) return true;
  (void)fp32;
  return la == 2 && lb >= 1;  // (dp|p), (dp|d), (dd|p), (dd|d)
}

// (dd|s): the cooperative kernel split over the orbital components.
inline bool eri3c_use_coop_a(int la, int lb) {
  const char *e = std::getenv("DFJK_ERI_COOP");
  if (e && e[0] == '0') return false;
  return la == 2 && lb == 2;
}

template <int LC>
struct CoopShape {
  static constexpr int G = ncart(LC);          // threads per aux shell
  static constexpr int SPW = 32 / G;           // aux shells per warp
  static constexpr int NW = LC == 2 ? 6 : 4;   // warps per block (static shared memory <= 48 KB)
  static constexpr int NS = NW * SPW;          // aux shells per block
  static constexpr int THREADS = NW * 32;
};

template <int LA, int LB, int LC, typename Real>
__global__ void __launch_bounds__(CoopShape<LC>::THREADS, 1) eri3c_coop_kernel(Eri3cArgs args, AuxArgs aux,
                                                                            const Real *__restrict__ boys_tab) {
  using Sh = CoopShape<LC>;
  constexpr int G = Sh::G, SPW = Sh::SPW, NS = Sh::NS;
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB);
  constexpr int LAB = LA + LB, L = LA + LB + LC;
  constexpr int NR = ntuv(L);
  __shared__ Real srec[REC];
  __shared__ double sP[3];
  __shared__ Real Rbuf[2][NS][NR];
  __shared__ int srt[NR];  // recursion table of the entries this kernel uses
  for (int i = threadIdx.x; i < NR; i += blockDim.x) srt[i] = c_rec.e[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / G, cc = lane - g * G;  // aux shell within the warp, aux component
  const bool lane_used = lane < SPW * G;
  const int slot = warp * SPW + (lane_used ? g : 0);  // aux shell within the block
  const int as = blockIdx.y * NS + slot;
  const bool active = lane_used && as < args.naux_shells;
  const int sc = active ? args.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  // this thread's aux component: a power 2 along one axis (xx, yy, zz) or
  // powers 1 (p, and xy, xz, yz)
  const int cx = cart_x(LC, cc), cy = cart_y(LC, cc), cz = cart_z(LC, cc);
  const int two = (cx == 2) ? 0 : (cy == 2) ? 1 : (cz == 2) ? 2 : -1;
  // shift of the W index: 2 along the doubled axis (xx, yy, zz), else the powers
  const int sh_y = two >= 0 ? (two == 1 ? 2 : 0) : cy, sh_z = two >= 0 ? (two == 2 ? 2 : 0) : cz;
  const int sh_yz = sh_y + sh_z;
  Real acc[NCA * NCB];
#pragma unroll
  for (int i = 0; i < NCA * NCB; ++i) acc[i] = Real(0);
  const double *rec0 = args.rec + args.rec_off[args.pairs[blockIdx.x]];
  const int npp = args.npp[args.pairs[blockIdx.x]];
  // every thread of the warp runs the same number of primitive iterations
  // (aux shells of a class share nprim here; nc is uniform within a group and
  // the warp-wide maximum bounds the loop)
  int ncmax = nc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ncmax = max(ncmax, __shfl_xor_sync(0xffffffffu, ncmax, o));
  for (int ipp = 0; ipp < npp; ++ipp) {
    __syncthreads();
    for (int i = threadIdx.x; i < REC; i += blockDim.x) {
      const double v = rec0[(long long)ipp * REC + i];
      srec[i] = (Real)v;
      if (i >= 1 && i <= 3) sP[i - 1] = v;
    }
    __syncthreads();
    for (int kc = 0; kc < ncmax; ++kc) {
      const bool live = kc < nc;
      const Real gexp = live ? (Real)aux.exps[pc0 + kc] : Real(1);
      const Real g1 = live ? (Real)aux.g1[pc0 + kc] : Real(0);
      const Real p = srec[0];
      // pair-to-aux-centre vector formed in FP64 before any rounding
      const Real X = (Real)(sP[0] - Cx), Y = (Real)(sP[1] - Cy), Z = (Real)(sP[2] - Cz);
      const Real sr = rsq(p + gexp);
      const Real al = p * gexp * (sr * sr);
      Real F[L + 1];
      boys_eval<L>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
      // R^(n), n = L .. 0, level by level in shared memory; R^(L) has one entry
      Real *cur = Rbuf[0][slot], *nxt = Rbuf[1][slot];
      Real pw = Real(1);
#pragma unroll
      for (int n = 0; n < L; ++n) pw *= Real(-2) * al;
      if (lane_used && cc == 0) cur[0] = pw * F[L];
      __syncwarp();
#pragma unroll
      for (int n = L - 1; n >= 0; --n) {
        pw = Real(1);
#pragma unroll
        for (int q = 0; q < n; ++q) pw *= Real(-2) * al;
        const int cnt = ntuv(L - n);
        if (lane_used)
          for (int k = cc; k < cnt; k += G) {
            Real r;
            if (k == 0) {
              r = pw * F[n];
            } else {
              const int e = srt[k];
              const int d = (e >> 16) & 3;
              const Real P = d == 0 ? X : (d == 1 ? Y : Z);
              r = fma(Real((e >> 18) & 15), cur[(e >> 8) & 255], P * cur[e & 255]);
            }
            nxt[k] = r;
          }
        __syncwarp();
        Real *tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
      // cur = R^(0); W for this thread's aux component (t + u + v <= LAB) is
      // read from it term by term in the contraction
      // W_tuv = c1 R_{t+dx, u+dy, v+dz} + c2 R_tuv with the shift of this
      // lane's component (dx + dy + dz = LC): xx-type c1 = 1/(2 gamma), c2 = 1;
      // xy-type and p c1 = 1, c2 = 0.  Branch-free, so the lanes of the
      // different components of a warp do not diverge.
      const Real *Rs = cur;
      const Real c1 = two >= 0 ? g1 : Real(1), c2 = two >= 0 ? Real(1) : Real(0);
      auto wval = [&](int t, int u, int v) -> Real {
        const int n1 = t + u + v + LC;                 // level of the shifted index
        const int s1 = u + v + sh_yz;                  // (u + dy) + (v + dz)
        const int i1 = n1 * (n1 + 1) * (n1 + 2) / 6 + s1 * (s1 + 1) / 2 + v + sh_z;
        if (LC == 1) return Rs[i1];                    // p: W = R shifted, c1 = 1, c2 = 0
        return fma(c1, Rs[i1], c2 * Rs[tuv_idx(t, u, v)]);
      };
      const Real scale = (two >= 0) ? g1 : (LC == 1 ? -g1 : g1 * g1);
      const Real ps = live ? srec[4] * (Real)aux.cdiv[pc0 + kc] * sr * scale : Real(0);
      int k = 0;
#pragma unroll
      for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
        for (int cb = 0; cb < NCB; ++cb) {
          const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
          const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
          Real sum = Real(0);
#pragma unroll
          for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
            for (int u = 0; u <= ay + by; ++u)
#pragma unroll
              for (int v = 0; v <= az + bz; ++v) sum = fma(srec[REC_HDR + k++], wval(t, u, v), sum);
          acc[ca * NCB + cb] = fma(ps, sum, acc[ca * NCB + cb]);
        }
      __syncwarp();  // R reads done before the next aux primitive overwrites it
    }
  }
  if (!active) return;
  const long long col0 = args.pair_col[args.pairs[blockIdx.x]] - args.col_begin;
  const int P = aux.func_off[sc] + cc;
  const double fc = comp_factor(LC, cc);
#pragma unroll
  for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb)
      args.T[(col0 + ca * NCB + cb) * args.ldT + P] =
          (double)acc[ca * NCB + cb] * (comp_factor(LA, ca) * comp_factor(LB, cb) * fc);
}

// The cooperative scheme for s aux functions (LC = 0), split over the
// components of the first orbital shell instead: the ncart(LA) threads of an
// aux shell share R (W = R for an s function) and each contracts it with the
// NCB component pairs of its own component a.  Used for (dd|s), whose
// one-thread kernel spills (ncu at 20 atoms: FP64 pipe 31 % busy).
template <int LA>
struct CoopShapeA {
  static constexpr int G = ncart(LA);
  static constexpr int SPW = 32 / G;
  static constexpr int NW = 4;
  static constexpr int NS = NW * SPW;
  static constexpr int THREADS = NW * 32;
};

template <int LA, int LB, typename Real>
__global__ void __launch_bounds__(CoopShapeA<LA>::THREADS, 1) eri3c_coop_a_kernel(Eri3cArgs args, AuxArgs aux,
                                                                                   const Real *__restrict__ boys_tab) {
  using Sh = CoopShapeA<LA>;
  constexpr int G = Sh::G, SPW = Sh::SPW, NS = Sh::NS;
  constexpr int NT = nterms(LA, LB);
  constexpr int REC = REC_HDR + NT;
  constexpr int NCA = ncart(LA), NCB = ncart(LB);
  constexpr int L = LA + LB;
  constexpr int NR = ntuv(L);
  __shared__ Real srec[REC];
  __shared__ double sP[3];
  __shared__ Real Rbuf[2][NS][NR];
  __shared__ int srt[NR];
  for (int i = threadIdx.x; i < NR; i += blockDim.x) srt[i] = c_rec.e[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / G, ca = lane - g * G;
  const bool lane_used = lane < SPW * G;
  const int slot = warp * SPW + (lane_used ? g : 0);
  const int as = blockIdx.y * NS + slot;
  const bool active = lane_used && as < args.naux_shells;
  const int sc = active ? args.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  // first term of component a's block in a primitive-pair record, and the
  // (t, u, v) ranges of each of its component pairs
  const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
  int k0 = 0;
#pragma unroll
  for (int a = 0; a < NCA; ++a)
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb)
      if (a < ca)
        k0 += (cart_x(LA, a) + cart_x(LB, cb) + 1) * (cart_y(LA, a) + cart_y(LB, cb) + 1) *
              (cart_z(LA, a) + cart_z(LB, cb) + 1);
  Real acc[NCB];
#pragma unroll
  for (int i = 0; i < NCB; ++i) acc[i] = Real(0);
  const double *rec0 = args.rec + args.rec_off[args.pairs[blockIdx.x]];
  const int npp = args.npp[args.pairs[blockIdx.x]];
  int ncmax = nc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ncmax = max(ncmax, __shfl_xor_sync(0xffffffffu, ncmax, o));
  for (int ipp = 0; ipp < npp; ++ipp) {
    __syncthreads();
    for (int i = threadIdx.x; i < REC; i += blockDim.x) {
      const double v = rec0[(long long)ipp * REC + i];
      srec[i] = (Real)v;
      if (i >= 1 && i <= 3) sP[i - 1] = v;
    }
    __syncthreads();
    for (int kc = 0; kc < ncmax; ++kc) {
      const bool live = kc < nc;
      const Real gexp = live ? (Real)aux.exps[pc0 + kc] : Real(1);
      const Real p = srec[0];
      const Real X = (Real)(sP[0] - Cx), Y = (Real)(sP[1] - Cy), Z = (Real)(sP[2] - Cz);
      const Real sr = rsq(p + gexp);
      const Real al = p * gexp * (sr * sr);
      Real F[L + 1];
      boys_eval<L>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
      Real *cur = Rbuf[0][slot], *nxt = Rbuf[1][slot];
      Real pw = Real(1);
#pragma unroll
      for (int n = 0; n < L; ++n) pw *= Real(-2) * al;
      if (lane_used && ca == 0) cur[0] = pw * F[L];
      __syncwarp();
#pragma unroll
      for (int n = L - 1; n >= 0; --n) {
        pw = Real(1);
#pragma unroll
        for (int q = 0; q < n; ++q) pw *= Real(-2) * al;
        const int cnt = ntuv(L - n);
        if (lane_used)
          for (int k = ca; k < cnt; k += G) {
            Real r;
            if (k == 0) {
              r = pw * F[n];
            } else {
              const int e = srt[k];
              const int d = (e >> 16) & 3;
              const Real P = d == 0 ? X : (d == 1 ? Y : Z);
              r = fma(Real((e >> 18) & 15), cur[(e >> 8) & 255], P * cur[e & 255]);
            }
            nxt[k] = r;
          }
        __syncwarp();
        Real *tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
      const Real ps = live ? srec[4] * (Real)aux.cdiv[pc0 + kc] * sr : Real(0);
      // this thread's component a: the (t, u, v) bounds depend on a at run
      // time, so the terms are walked with runtime loops over small ranges
      int k = k0;
#pragma unroll
      for (int cb = 0; cb < NCB; ++cb) {
        const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
        Real sum = Real(0);
        for (int t = 0; t <= ax + bx; ++t)
          for (int u = 0; u <= ay + by; ++u)
            for (int v = 0; v <= az + bz; ++v) sum = fma(srec[REC_HDR + k++], cur[tuv_idx_rt(t, u, v)], sum);
        acc[cb] = fma(ps, sum, acc[cb]);
      }
      __syncwarp();
    }
  }
  if (!active) return;
  const long long col0 = args.pair_col[args.pairs[blockIdx.x]] - args.col_begin;
  const int P = aux.func_off[sc];
  const double fa = comp_factor(LA, ca);
#pragma unroll
  for (int cb = 0; cb < NCB; ++cb)
    args.T[(col0 + ca * NCB + cb) * args.ldT + P] = (double)acc[cb] * (fa * comp_factor(LB, cb));
}

// ---- 2-centre metric and overlap ----------------------------------------------

// Hermite expansion of a one-centre Cartesian power k with exponent a, one
// direction: up to two terms (t, coefficient).
__device__ __forceinline__ int one_centre_terms(int k, double inv2a, int *t, double *c) {
  if (k == 0) {
    t[0] = 0; c[0] = 1.0;
    return 1;
  }
  if (k == 1) {
    t[0] = 1; c[0] = inv2a;
    return 1;
  }
  t[0] = 0; c[0] = inv2a;
  t[1] = 2; c[1] = inv2a * inv2a;
  return 2;
}

// One thread per aux shell pair (P >= Q in internal order, class (LP, LQ)).
template <int LP, int LQ>
__global__ void __launch_bounds__(128) metric_kernel(MetricArgs args, AuxArgs aux,
                                                     const double *__restrict__ boys_tab) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= args.npair) return;
  constexpr int L = LP + LQ;
  constexpr int NP = ncart(LP), NQ = ncart(LQ);
  const int sp = args.shell_p[ip], sq = args.shell_q[ip];
  const double X = aux.center[3 * sp] - aux.center[3 * sq];
  const double Y = aux.center[3 * sp + 1] - aux.center[3 * sq + 1];
  const double Z = aux.center[3 * sp + 2] - aux.center[3 * sq + 2];
  double out[NP * NQ];
#pragma unroll
  for (int i = 0; i < NP * NQ; ++i) out[i] = 0.0;
  for (int kp = 0; kp < aux.nprim[sp]; ++kp)
    for (int kq = 0; kq < aux.nprim[sq]; ++kq) {
      const int ip0 = aux.prim_off[sp] + kp, iq0 = aux.prim_off[sq] + kq;
      const double a = aux.exps[ip0], g = aux.exps[iq0];
      const double s = rsqrt(a + g);
      const double al = a * g * s * s;
      double F[L + 1];
      boys_eval<L>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
      double R[ntuv(L)];
      hermite_R<L>(F, al, X, Y, Z, R);
      // 2 pi^2.5/(a g sqrt(a+g)) c_a c_g = 2 pi^2.5 s cdiv_a cdiv_g
      const double pref = 2.0 * 17.493418327624862846 * s * aux.cdiv[ip0] * aux.cdiv[iq0];
#pragma unroll
      for (int cp = 0; cp < NP; ++cp)
#pragma unroll
        for (int cq = 0; cq < NQ; ++cq) {
          int tp[3][2], tq[3][2], np_[3], nq_[3];
          double cpf[3][2], cqf[3][2];
          np_[0] = one_centre_terms(cart_x(LP, cp), aux.g1[ip0], tp[0], cpf[0]);
          np_[1] = one_centre_terms(cart_y(LP, cp), aux.g1[ip0], tp[1], cpf[1]);
          np_[2] = one_centre_terms(cart_z(LP, cp), aux.g1[ip0], tp[2], cpf[2]);
          nq_[0] = one_centre_terms(cart_x(LQ, cq), aux.g1[iq0], tq[0], cqf[0]);
          nq_[1] = one_centre_terms(cart_y(LQ, cq), aux.g1[iq0], tq[1], cqf[1]);
          nq_[2] = one_centre_terms(cart_z(LQ, cq), aux.g1[iq0], tq[2], cqf[2]);
          double sum = 0.0;
          for (int i0 = 0; i0 < np_[0]; ++i0)
            for (int i1 = 0; i1 < np_[1]; ++i1)
              for (int i2 = 0; i2 < np_[2]; ++i2)
                for (int j0 = 0; j0 < nq_[0]; ++j0)
                  for (int j1 = 0; j1 < nq_[1]; ++j1)
                    for (int j2 = 0; j2 < nq_[2]; ++j2) {
                      const int t = tp[0][i0] + tq[0][j0], u = tp[1][i1] + tq[1][j1],
                                v = tp[2][i2] + tq[2][j2];
                      const double sg = ((tq[0][j0] + tq[1][j1] + tq[2][j2]) & 1) ? -1.0 : 1.0;
                      sum += sg * cpf[0][i0] * cpf[1][i1] * cpf[2][i2] * cqf[0][j0] * cqf[1][j1] *
                             cqf[2][j2] * R[tuv_idx(t, u, v)];
                    }
          out[cp * NQ + cq] += pref * sum;
        }
    }
  const int P0 = aux.func_off[sp], Q0 = aux.func_off[sq];
  for (int cp = 0; cp < NP; ++cp)
    for (int cq = 0; cq < NQ; ++cq) {
      const double v = out[cp * NQ + cq] * comp_factor(LP, cp) * comp_factor(LQ, cq);
      args.V[(long long)(P0 + cp) * args.ldV + Q0 + cq] = v;
      args.V[(long long)(Q0 + cq) * args.ldV + P0 + cp] = v;
    }
}

// Overlap <a|b> = sum c_a c_b K_ab (pi/p)^(3/2) E^x_0 E^y_0 E^z_0; one thread
// per ordered orbital shell pair.
template <int LA, int LB>
__global__ void overlap_kernel(OverlapArgs args, OrbArgs orb) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= args.npair) return;
  constexpr int NCA = ncart(LA), NCB = ncart(LB);
  const int sa = args.shell_a[ip], sb = args.shell_b[ip];
  const double Ax = orb.center[3 * sa], Ay = orb.center[3 * sa + 1], Az = orb.center[3 * sa + 2];
  const double Bx = orb.center[3 * sb], By = orb.center[3 * sb + 1], Bz = orb.center[3 * sb + 2];
  const double AB2 = (Ax - Bx) * (Ax - Bx) + (Ay - By) * (Ay - By) + (Az - Bz) * (Az - Bz);
  double out[NCA * NCB];
#pragma unroll
  for (int i = 0; i < NCA * NCB; ++i) out[i] = 0.0;
  for (int ka = 0; ka < orb.nprim[sa]; ++ka)
    for (int kb = 0; kb < orb.nprim[sb]; ++kb) {
      const double a = orb.exps[orb.prim_off[sa] + ka], b = orb.exps[orb.prim_off[sb] + kb];
      const double p = a + b, ip_ = 1.0 / p;
      const double Px = (a * Ax + b * Bx) * ip_, Py = (a * Ay + b * By) * ip_,
                   Pz = (a * Az + b * Bz) * ip_;
      double Ex[LA + 1][LB + 1][LA + LB + 1], Ey[LA + 1][LB + 1][LA + LB + 1],
          Ez[LA + 1][LB + 1][LA + LB + 1];
      hermite_E<LA, LB>(0.5 * ip_, Px - Ax, Px - Bx, Ex);
      hermite_E<LA, LB>(0.5 * ip_, Py - Ay, Py - By, Ey);
      hermite_E<LA, LB>(0.5 * ip_, Pz - Az, Pz - Bz, Ez);
      const double pref = orb.coefs[orb.prim_off[sa] + ka] * orb.coefs[orb.prim_off[sb] + kb] *
                          exp(-a * b * ip_ * AB2) * (5.5683279968317078453 * ip_ * sqrt(ip_));
#pragma unroll
      for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
        for (int cb = 0; cb < NCB; ++cb)
          out[ca * NCB + cb] += pref * Ex[cart_x(LA, ca)][cart_x(LB, cb)][0] *
                                Ey[cart_y(LA, ca)][cart_y(LB, cb)][0] *
                                Ez[cart_z(LA, ca)][cart_z(LB, cb)][0];
    }
  const int A0 = orb.func_off[sa], B0 = orb.func_off[sb];
  for (int ca = 0; ca < NCA; ++ca)
    for (int cb = 0; cb < NCB; ++cb) {
      const double v = out[ca * NCB + cb] * comp_factor(LA, ca) * comp_factor(LB, cb);
      args.S[(long long)(A0 + ca) * args.ldS + B0 + cb] = v;
      args.S[(long long)(B0 + cb) * args.ldS + A0 + ca] = v;
    }
}

// Boys table evaluation for tests.
template <int M>
__global__ void boys_kernel(int n, const double *__restrict__ T, double *__restrict__ F,
                            const double *__restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[M + 1];
  boys_eval<M>(T[i], tab, f);
  for (int m = 0; m <= M; ++m) F[(long long)i * (M + 1) + m] = f[m];
}


#define DISPATCH_LALB(LA, LB, CALL)                                   \
  switch ((LA) * 3 + (LB)) {                                          \
    case 0: { constexpr int A_ = 0, B_ = 0; CALL; } break;            \
    case 3: { constexpr int A_ = 1, B_ = 0; CALL; } break;            \
    case 4: { constexpr int A_ = 1, B_ = 1; CALL; } break;            \
    case 6: { constexpr int A_ = 2, B_ = 0; CALL; } break;            \
    case 7: { constexpr int A_ = 2, B_ = 1; CALL; } break;            \
    case 8: { constexpr int A_ = 2, B_ = 2; CALL; } break;            \
    default: throw Error{DFJK_ERR_UNSUPPORTED, "shell class"};        \
  }

}  // namespace dfjk
