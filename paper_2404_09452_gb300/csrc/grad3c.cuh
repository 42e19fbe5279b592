// Derivative 3-centre kernel of the DF Coulomb/exchange gradient, shared by the
// per-aux-class translation units grad3c_l{0,1,2}.cu (split so that they
// compile in parallel).  The scheme is described in grad.cu.
#pragma once

#include "grad.cuh"
#include "md.cuh"

namespace dfjk {

// (t, u, v) of a dense Hermite index (the inverse of tuv_idx).
__device__ __forceinline__ void tuv_decode(int idx, int &t, int &u, int &v) {
  int N = 0;
  while (ntuv(N) <= idx) ++N;
  int r = idx - (N > 0 ? ntuv(N - 1) : 0), sl = 0;
  while ((sl + 1) * (sl + 2) / 2 <= r) ++sl;
  v = r - sl * (sl + 1) / 2;
  u = sl - v;
  t = N - sl;
}

// Exchange weights, one (ca, cb) component pair at a time, every loop unrolled
// at compile time so that W stays in registers: dA_q = sum_tuv E1_q E0 E0 W,
// dC_q = -sum_tuv E0 E0 E0 W[tuv + 1_q].  The sums are taken as
// sum_t E_x sum_u E_y (sum_v E_z W): the v contractions (plain, raised, and
// against the three shifted W) first, then the (t, u) lines.
template <int LA, int LB, int NT>
__device__ __forceinline__ void k_weights(const double (*sE)[LA + 2][LB + 1][LA + LB + 2],
                                          const double (*sR1)[LA + 1][LB + 1][LA + LB + 2], const double *W,
                                          const double *__restrict__ Gp, long long nao, double wk, double *gA,
                                          double *gCp) {
  constexpr int NCA = ncart(LA), NCB = ncart(LB), LAB = LA + LB;
#pragma unroll
  for (int ca = 0; ca < NCA; ++ca)
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb) {
      const int ax = cart_x(LA, ca), ay = cart_y(LA, ca), az = cart_z(LA, ca);
      const int bx = cart_x(LB, cb), by = cart_y(LB, cb), bz = cart_z(LB, cb);
      const double wt = wk * __ldg(Gp + ca * nao + cb) * (comp_factor(LA, ca) * comp_factor(LB, cb));
      double dA0 = 0.0, dA1 = 0.0, dA2 = 0.0, dC0 = 0.0, dC1 = 0.0, dC2 = 0.0;
#pragma unroll
      for (int t = 0; t <= ax + bx + 1; ++t)
#pragma unroll
        for (int u = 0; u <= ay + by + 1; ++u) {
          if (t + u > LAB + 1) continue;
          const bool in_x = t <= ax + bx, in_y = u <= ay + by;
          if (!in_x && !in_y) continue;  // no term has both raised
          double vz0 = 0.0, vz1 = 0.0, vsx = 0.0, vsy = 0.0, vsz = 0.0;
#pragma unroll
          for (int v = 0; v <= az + bz + 1; ++v) {
            if (t + u + v > LAB + 1) continue;
            const double w = W[tuv_idx(t, u, v)];
            const double e1z = sR1[2][az][bz][v];
            if (in_x && in_y) vz1 = fma(e1z, w, vz1);
            if (v <= az + bz) {
              const double e0z = sE[2][az][bz][v];
              vz0 = fma(e0z, w, vz0);
              if (in_x && in_y) {
                vsx = fma(e0z, W[tuv_idx(t + 1, u, v)], vsx);
                vsy = fma(e0z, W[tuv_idx(t, u + 1, v)], vsy);
                vsz = fma(e0z, W[tuv_idx(t, u, v + 1)], vsz);
              }
            }
          }
          const double e0x = in_x ? sE[0][ax][bx][t] : 0.0, e1x = sR1[0][ax][bx][t];
          const double e0y = in_y ? sE[1][ay][by][u] : 0.0, e1y = sR1[1][ay][by][u];
          if (in_y) dA0 = fma(e1x * e0y, vz0, dA0);
          if (in_x) dA1 = fma(e0x * e1y, vz0, dA1);
          if (in_x && in_y) {
            const double exy = e0x * e0y;
            dA2 = fma(exy, vz1, dA2);
            dC0 = fma(-exy, vsx, dC0);
            dC1 = fma(-exy, vsy, dC1);
            dC2 = fma(-exy, vsz, dC2);
          }
        }
      gA[0] = fma(wt, dA0, gA[0]);
      gA[1] = fma(wt, dA1, gA[1]);
      gA[2] = fma(wt, dA2, gA[2]);
      gCp[0] = fma(wt, dC0, gCp[0]);
      gCp[1] = fma(wt, dC1, gCp[1]);
      gCp[2] = fma(wt, dC2, gCp[2]);
    }
}

// W[tuv] = sum over the Hermite terms of aux component cc of
// (-1)^(t'+u'+v') coef R[t + t', u + u', v + v'], for t + u + v <= LAB + 1.
template <int LAB, int LC, typename Real>
__device__ __forceinline__ void aux_w(int cc, double g1, const Real *R, Real *W) {
  int tc[3][2];
  double fc[3][2];
  const int n0 = one_centre_terms(cart_x(LC, cc), g1, tc[0], fc[0]);
  const int n1 = one_centre_terms(cart_y(LC, cc), g1, tc[1], fc[1]);
  const int n2 = one_centre_terms(cart_z(LC, cc), g1, tc[2], fc[2]);
#pragma unroll
  for (int N = 0; N <= LAB + 1; ++N)
#pragma unroll
    for (int t = N; t >= 0; --t)
#pragma unroll
      for (int u = N - t; u >= 0; --u) {
        const int v = N - t - u;
        Real w = Real(0);
        for (int i0 = 0; i0 < n0; ++i0)
          for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n2; ++i2) {
              const int ts = tc[0][i0] + tc[1][i1] + tc[2][i2];
              const double c = fc[0][i0] * fc[1][i1] * fc[2][i2] * ((ts & 1) ? -1.0 : 1.0);
              w = fma(Real(c), R[tuv_idx(t + tc[0][i0], u + tc[1][i1], v + tc[2][i2])], w);
            }
        W[tuv_idx(t, u, v)] = w;
      }
}

// Coulomb weights alone, one aux primitive: Boys, R, the aux components' W
// summed with their weights cj d_P (times the prefactor), then one set of dot
// products with the block's HA_q / H0.  Real = float for the shell pairs whose
// integrals the build also evaluates in FP32 (Schwarz bound below the FP32
// threshold); the sums over terms are added to FP64 accumulators.
template <int LAB, int LC, int L1, typename Real>
__device__ __forceinline__ void coulomb_alone(double al, double X, double Y, double Z, double pt, double g1,
                                              const double *dP, const double *sHA, const double *sH0,
                                              const Real *tab, double *gA, double *gCp) {
  constexpr int NT1 = ntuv(LAB + 1), NCC = ncart(LC);
  Real F[L1 + 1];
  boys_eval<L1>(Real(al * (X * X + Y * Y + Z * Z)), tab, F);
  Real R[ntuv(L1)];
  hermite_R<L1, Real>(F, Real(al), Real(X), Real(Y), Real(Z), R);
  Real Ws[NT1];
#pragma unroll
  for (int e = 0; e < NT1; ++e) Ws[e] = Real(0);
#pragma unroll 1
  for (int cc = 0; cc < NCC; ++cc) {
    Real W[NT1];
    aux_w<LAB, LC, Real>(cc, g1, R, W);
    const Real sj = Real(pt * comp_factor(LC, cc) * dP[cc]);
#pragma unroll
    for (int e = 0; e < NT1; ++e) Ws[e] = fma(sj, W[e], Ws[e]);
  }
  Real hA0 = 0, hA1 = 0, hA2 = 0, hC0 = 0, hC1 = 0, hC2 = 0;
#pragma unroll
  for (int e = 0; e < NT1; ++e) {
    hA0 = fma(Real(sHA[e]), Ws[e], hA0);
    hA1 = fma(Real(sHA[NT1 + e]), Ws[e], hA1);
    hA2 = fma(Real(sHA[2 * NT1 + e]), Ws[e], hA2);
  }
#pragma unroll
  for (int N = 0; N <= LAB; ++N)
#pragma unroll
    for (int t = N; t >= 0; --t)
#pragma unroll
      for (int u = N - t; u >= 0; --u) {
        const int v = N - t - u;
        const Real h0 = Real(sH0[tuv_idx(t, u, v)]);
        hC0 = fma(h0, Ws[tuv_idx(t + 1, u, v)], hC0);
        hC1 = fma(h0, Ws[tuv_idx(t, u + 1, v)], hC1);
        hC2 = fma(h0, Ws[tuv_idx(t, u, v + 1)], hC2);
      }
  gA[0] += double(hA0);
  gA[1] += double(hA1);
  gA[2] += double(hA2);
  gCp[0] -= double(hC0);
  gCp[1] -= double(hC1);
  gCp[2] -= double(hC2);
}

// Block: pair_chunk kept pairs of class (LA, LB) (one in practice) x 128 aux
// shells of class LC, a thread per aux shell.  The Coulomb weights
// cj d_P D_mu nu factor into an aux part and a pair part, so the pair part is
// contracted with the Hermite coefficients once per primitive pair (shared
// memory, all threads): HA_q[tuv] = sum_{ab} D_ab dE_ab/dA_q [tuv] and
// H0[tuv] = sum_{ab} D_ab E_ab[tuv]; each thread then needs dot products with
// its W.  The exchange weights (gam, EXCH) differ per aux function and run
// component by component.  F32: the Coulomb-only per-thread part in FP32.
template <int LA, int LB, int LC, bool EXCH, bool F32>
__global__ void __launch_bounds__(128, 2) grad3c_kernel(GradArgs g, OrbArgs orb, AuxArgs aux,
                                                        const double *__restrict__ boys_tab,
                                                        const float *__restrict__ boys_tab32) {
  constexpr int NCA = ncart(LA), NCB = ncart(LB), NCC = ncart(LC);
  constexpr int LAB = LA + LB, L1 = LA + LB + LC + 1;
  constexpr int EI = LA + 2, EJ = LB + 1, ET = LA + LB + 2;  // E[i <= LA+1][j <= LB][t <= LAB+1]
  constexpr int NT1 = ntuv(LAB + 1), NT0 = ntuv(LAB);
  // tables of up to KK primitive pairs at a time (one barrier round per group)
  constexpr int KK = 4, NH = 3 * NT1 + NT0;
  __shared__ double sE[KK][3][EI][EJ][ET];
  __shared__ double sR1[KK][3][LA + 1][EJ][ET];  // 2 alpha E^{i+1, j} - i E^{i-1, j}
  __shared__ double sHdr[KK][6];                 // 2 alpha, prefactor, Px, Py, Pz
  __shared__ double sD[NCA * NCB];
  __shared__ double sHA[KK][3][NT1], sH0[KK][NT0];
  __shared__ double sRed[4][6];
  const bool cj_on = g.cj != 0.0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int as = blockIdx.y * blockDim.x + tid;
  const bool active = as < g.naux_shells;
  const int sc = active ? g.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  double dP[NCC];
#pragma unroll
  for (int cc = 0; cc < NCC; ++cc) dP[cc] = active ? g.cj * g.d[aux.func_off[sc] + cc] : 0.0;
  const long long nao2 = (long long)g.nao * g.nao;
  // EXCH: exchange weights present (g.gam); a separate instantiation keeps the
  // Coulomb-only kernel's registers free of the exchange loop
  const double *gP = EXCH ? g.gam + (long long)(active ? aux.func_off[sc] : 0) * nao2 : nullptr;
  double gC[3] = {0.0, 0.0, 0.0};
  const int p0 = blockIdx.x * g.pair_chunk, p1 = min(g.npairs, p0 + g.pair_chunk);
#pragma unroll 1
  for (int ip = p0; ip < p1; ++ip) {
    const int pair = g.pairs[ip];
    const int sa = g.pair_a[pair], sb = g.pair_b[pair];
    const int mu0 = orb.func_off[sa], nu0 = orb.func_off[sb];
    const double kf = g.ck * (sa == sb ? 1.0 : 2.0);
    __syncthreads();
    if (tid < NCA * NCB) {
      const int mu = mu0 + tid / NCB, nu = nu0 + tid % NCB;
      sD[tid] = g.D[(long long)mu * g.nao + nu] * (sa == sb ? 1.0 : 2.0);
    }
    const double Ax = orb.center[3 * sa], Ay = orb.center[3 * sa + 1], Az = orb.center[3 * sa + 2];
    const double Bx = orb.center[3 * sb], By = orb.center[3 * sb + 1], Bz = orb.center[3 * sb + 2];
    const double AB2 = (Ax - Bx) * (Ax - Bx) + (Ay - By) * (Ay - By) + (Az - Bz) * (Az - Bz);
    const int pa0 = orb.prim_off[sa], na = orb.nprim[sa], pb0 = orb.prim_off[sb], nb = orb.nprim[sb];
    double gA[3] = {0.0, 0.0, 0.0}, gCp[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int k0 = 0; k0 < na * nb; k0 += KK) {
      const int cnt = min(KK, na * nb - k0);
      __syncthreads();
      if (tid < 3 * cnt) {  // one thread per (primitive pair, direction) builds its tables
        const int k = tid / 3, dir = tid % 3, kk = k0 + k;
        const int ka = kk / nb, kb = kk % nb;
        const double a = orb.exps[pa0 + ka], b = orb.exps[pb0 + kb], p = a + b, ip_ = 1.0 / p;
        const double A = dir == 0 ? Ax : dir == 1 ? Ay : Az, Bc = dir == 0 ? Bx : dir == 1 ? By : Bz;
        const double P = (a * A + b * Bc) * ip_;
        double E[EI][EJ][ET];
        hermite_E<LA + 1, LB>(0.5 * ip_, P - A, P - Bc, E);
#pragma unroll
        for (int i = 0; i < EI; ++i)
#pragma unroll
          for (int j = 0; j < EJ; ++j)
#pragma unroll
            for (int t = 0; t < ET; ++t) {
              sE[k][dir][i][j][t] = E[i][j][t];
              if (i <= LA) sR1[k][dir][i][j][t] = 2.0 * a * E[i + 1][j][t] - (i > 0 ? i * E[i - 1][j][t] : 0.0);
            }
        sHdr[k][2 + dir] = P;
        if (dir == 0) {
          sHdr[k][0] = 2.0 * a;
          sHdr[k][1] = orb.coefs[pa0 + ka] * orb.coefs[pb0 + kb] * exp(-a * b * ip_ * AB2) *
                       (2.0 * 17.493418327624862846 * ip_);  // c_a c_b K_ab 2 pi^(5/2) / p
        }
      }
      __syncthreads();
      if (cj_on) {  // Coulomb weights contracted with the Hermite coefficients
        for (int ek = tid; ek < cnt * NH; ek += blockDim.x) {
          const int k = ek / NH, e = ek % NH;
          const int q = e < 3 * NT1 ? e / NT1 : 3;
          int tt[3];
          tuv_decode(q < 3 ? e - q * NT1 : e - 3 * NT1, tt[0], tt[1], tt[2]);
          double h = 0.0;
#pragma unroll 1
          for (int ca = 0; ca < NCA; ++ca)
#pragma unroll 1
            for (int cb = 0; cb < NCB; ++cb) {
              const int ax[3] = {cart_x(LA, ca), cart_y(LA, ca), cart_z(LA, ca)};
              const int bx[3] = {cart_x(LB, cb), cart_y(LB, cb), cart_z(LB, cb)};
              double f = sD[ca * NCB + cb] * comp_factor(LA, ca) * comp_factor(LB, cb);
              for (int r = 0; r < 3; ++r)
                f *= (r == q) ? sR1[k][r][ax[r]][bx[r]][tt[r]] : sE[k][r][ax[r]][bx[r]][tt[r]];
              h += f;
            }
          if (q < 3) sHA[k][q][e - q * NT1] = h;
          else sH0[k][e - 3 * NT1] = h;
        }
        __syncthreads();
      }
#pragma unroll 1
      for (int k = 0; k < cnt; ++k) {
        const double X = sHdr[k][2] - Cx, Y = sHdr[k][3] - Cy, Z = sHdr[k][4] - Cz;
        const int ka = (k0 + k) / nb, kb = (k0 + k) % nb;
        const double p = orb.exps[pa0 + ka] + orb.exps[pb0 + kb];
#pragma unroll 1
        for (int kc = 0; kc < nc; ++kc) {
          const double gm = aux.exps[pc0 + kc], g1 = aux.g1[pc0 + kc];
          const double s = rsqrt(p + gm);
          const double al = p * gm * (s * s);
          const double pt = sHdr[k][1] * aux.cdiv[pc0 + kc] * s;
          if (!EXCH) {  // Coulomb alone: sum_cc s_cc W_cc first, then one set of dot products
            if (cj_on) {
              if (F32)
                coulomb_alone<LAB, LC, L1, float>(al, X, Y, Z, pt, g1, dP, &sHA[k][0][0], sH0[k], boys_tab32, gA,
                                                  gCp);
              else
                coulomb_alone<LAB, LC, L1, double>(al, X, Y, Z, pt, g1, dP, &sHA[k][0][0], sH0[k], boys_tab, gA,
                                                   gCp);
            }
            continue;
          }
          double F[L1 + 1];
          boys_eval<L1>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
          double R[ntuv(L1)];
          hermite_R<L1>(F, al, X, Y, Z, R);
          if (EXCH) {  // exchange (and Coulomb, if on) per aux component
#pragma unroll 1
            for (int cc = 0; cc < NCC; ++cc) {
              double W[NT1];
              aux_w<LAB, LC>(cc, g1, R, W);
              const double wc = pt * comp_factor(LC, cc);
              if (cj_on) {
                const double sj = wc * dP[cc];
                double hA0 = 0.0, hA1 = 0.0, hA2 = 0.0, hC0 = 0.0, hC1 = 0.0, hC2 = 0.0;
#pragma unroll
                for (int e = 0; e < NT1; ++e) {
                  hA0 = fma(sHA[k][0][e], W[e], hA0);
                  hA1 = fma(sHA[k][1][e], W[e], hA1);
                  hA2 = fma(sHA[k][2][e], W[e], hA2);
                }
#pragma unroll
                for (int N = 0; N <= LAB; ++N)
#pragma unroll
                  for (int t = N; t >= 0; --t)
#pragma unroll
                    for (int u = N - t; u >= 0; --u) {
                      const int v = N - t - u;
                      const double h0 = sH0[k][tuv_idx(t, u, v)];
                      hC0 = fma(h0, W[tuv_idx(t + 1, u, v)], hC0);
                      hC1 = fma(h0, W[tuv_idx(t, u + 1, v)], hC1);
                      hC2 = fma(h0, W[tuv_idx(t, u, v + 1)], hC2);
                    }
                gA[0] = fma(sj, hA0, gA[0]);
                gA[1] = fma(sj, hA1, gA[1]);
                gA[2] = fma(sj, hA2, gA[2]);
                gCp[0] = fma(-sj, hC0, gCp[0]);
                gCp[1] = fma(-sj, hC1, gCp[1]);
                gCp[2] = fma(-sj, hC2, gCp[2]);
              }
              k_weights<LA, LB, NT1>(sE[k], sR1[k], W, gP + cc * nao2 + (long long)mu0 * g.nao + nu0, g.nao,
                                     wc * kf, gA, gCp);
            }
          }
        }
      }
    }
    // this pair: A and B = -(A + C) summed over the block's aux shells; C per thread
    double red[6];
    for (int q = 0; q < 3; ++q) {
      red[q] = gA[q];
      red[3 + q] = -(gA[q] + gCp[q]);
      gC[q] += gCp[q];
    }
    for (int q = 0; q < 6; ++q)
      for (int o = 16; o > 0; o >>= 1) red[q] += __shfl_xor_sync(0xffffffffu, red[q], o);
    if (lane == 0)
      for (int q = 0; q < 6; ++q) sRed[warp][q] = red[q];
    __syncthreads();
    if (tid < 6) {
      const double v = sRed[0][tid] + sRed[1][tid] + sRed[2][tid] + sRed[3][tid];
      const int atom = tid < 3 ? g.orb_atom[sa] : g.orb_atom[sb];
      atomicAdd(&g.grad[3 * atom + tid % 3], v);
    }
  }
  if (active)
    for (int q = 0; q < 3; ++q) atomicAdd(&g.grad[3 * g.aux_atom[sc] + q], gC[q]);
}

}  // namespace dfjk
