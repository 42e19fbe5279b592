// Nuclear gradient of the density-fitted Coulomb energy (FP64).
//
// E_J = u^T V^-1 u / 2 with u_P = sum_{mu nu} (P|mu nu) D_mu nu, so at fixed D
//   dE_J/dR = sum_P d_P du_P/dR - d^T (dV/dR) d / 2,   d = V^-1 u = L^-T rho,
// rho = L^-1 u = B vec(D) being the build's fitted vector.  Derivatives of the
// integrals, McMurchie-Davidson form:
//  * orbital centre A:  d/dA_x [x_A^i e^{-a x_A^2}] = 2a x_A^{i+1} e - i x_A^{i-1} e,
//    i.e. the E^{i+1, j} and E^{i-1, j} Hermite coefficients of the pair;
//  * one-centre (aux) Gaussian at C: d/dC_x Lambda_t = Lambda_{t+1}, a shift of
//    the Hermite index;
//  * the second orbital centre B by translational invariance, dB = -(dA + dC),
//    triple by triple.
// For the metric term only pairs on different atoms contribute (the
// derivatives of same-atom pairs cancel), each as -d_P d_Q d(P|Q)/dR_P on the
// atom of P.  Loops are runtime loops: this runs once per geometry, and
// unrolling the derivative classes (L up to 7) would cost minutes of compile.
#include "grad.cuh"
#include "md.cuh"

namespace dfjk {

// Block: a chunk of kept pairs of class (LA, LB) x 128 aux shells of class LC.
template <int LA, int LB, int LC>
__global__ void __launch_bounds__(128) grad3c_kernel(GradArgs g, OrbArgs orb, AuxArgs aux,
                                                     const double *__restrict__ boys_tab) {
  constexpr int NCA = ncart(LA), NCB = ncart(LB), NCC = ncart(LC);
  constexpr int LAB = LA + LB, L1 = LA + LB + LC + 1;
  constexpr int EI = LA + 2, EJ = LB + 1, ET = LA + LB + 2;  // E[i <= LA+1][j <= LB][t <= LAB+1]
  __shared__ double sE[3][EI][EJ][ET];
  __shared__ double sHdr[6];  // 2 alpha, prefactor, Px, Py, Pz
  __shared__ double sD[NCA * NCB];
  __shared__ double sRed[4][6];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int as = blockIdx.y * blockDim.x + tid;
  const bool active = as < g.naux_shells;
  const int sc = active ? g.aux_shells[as] : 0;
  const double Cx = aux.center[3 * sc], Cy = aux.center[3 * sc + 1], Cz = aux.center[3 * sc + 2];
  const int pc0 = aux.prim_off[sc], nc = active ? aux.nprim[sc] : 0;
  double dP[NCC];
  for (int cc = 0; cc < NCC; ++cc) dP[cc] = active ? g.cj * g.d[aux.func_off[sc] + cc] : 0.0;
  const long long nao2 = (long long)g.nao * g.nao;
  const double *gP = g.gam ? g.gam + (long long)(active ? aux.func_off[sc] : 0) * nao2 : nullptr;
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
      const int mu = orb.func_off[sa] + tid / NCB, nu = orb.func_off[sb] + tid % NCB;
      sD[tid] = g.D[(long long)mu * g.nao + nu] * (sa == sb ? 1.0 : 2.0);
    }
    const double Ax = orb.center[3 * sa], Ay = orb.center[3 * sa + 1], Az = orb.center[3 * sa + 2];
    const double Bx = orb.center[3 * sb], By = orb.center[3 * sb + 1], Bz = orb.center[3 * sb + 2];
    const double AB2 = (Ax - Bx) * (Ax - Bx) + (Ay - By) * (Ay - By) + (Az - Bz) * (Az - Bz);
    const int pa0 = orb.prim_off[sa], na = orb.nprim[sa], pb0 = orb.prim_off[sb], nb = orb.nprim[sb];
    double gA[3] = {0.0, 0.0, 0.0}, gCp[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int kk = 0; kk < na * nb; ++kk) {
      __syncthreads();
      if (tid < 3) {  // one thread per direction builds that direction's E table
        const int ka = kk / nb, kb = kk % nb;
        const double a = orb.exps[pa0 + ka], b = orb.exps[pb0 + kb], p = a + b, ip_ = 1.0 / p;
        const double A = tid == 0 ? Ax : tid == 1 ? Ay : Az, Bc = tid == 0 ? Bx : tid == 1 ? By : Bz;
        const double P = (a * A + b * Bc) * ip_;
        double E[EI][EJ][ET];
        hermite_E<LA + 1, LB>(0.5 * ip_, P - A, P - Bc, E);
        for (int i = 0; i < EI; ++i)
          for (int j = 0; j < EJ; ++j)
            for (int t = 0; t < ET; ++t) sE[tid][i][j][t] = E[i][j][t];
        sHdr[2 + tid] = P;
        if (tid == 0) {
          sHdr[0] = 2.0 * a;
          sHdr[1] = orb.coefs[pa0 + ka] * orb.coefs[pb0 + kb] * exp(-a * b * ip_ * AB2) *
                    (2.0 * 17.493418327624862846 * ip_);  // c_a c_b K_ab 2 pi^(5/2) / p
        }
      }
      __syncthreads();
      const double a2 = sHdr[0];
      const double X = sHdr[2] - Cx, Y = sHdr[3] - Cy, Z = sHdr[4] - Cz;
      const int ka = kk / nb, kb = kk % nb;
      const double p = orb.exps[pa0 + ka] + orb.exps[pb0 + kb];
#pragma unroll 1
      for (int kc = 0; kc < nc; ++kc) {
        const double gm = aux.exps[pc0 + kc], g1 = aux.g1[pc0 + kc];
        const double s = rsqrt(p + gm);
        const double al = p * gm * (s * s);
        double F[L1 + 1];
        boys_eval<L1>(al * (X * X + Y * Y + Z * Z), boys_tab, F);
        double R[ntuv(L1)];
        hermite_R<L1>(F, al, X, Y, Z, R);
        const double pt = sHdr[1] * aux.cdiv[pc0 + kc] * s;
#pragma unroll 1
        for (int cc = 0; cc < NCC; ++cc) {
          const int cx = cart_x(LC, cc), cy = cart_y(LC, cc), cz = cart_z(LC, cc);
          // aux Hermite terms (t, coefficient) per direction and their sign
          int tc[3][2];
          double fc[3][2];
          const int n0 = one_centre_terms(cx, g1, tc[0], fc[0]), n1 = one_centre_terms(cy, g1, tc[1], fc[1]),
                    n2 = one_centre_terms(cz, g1, tc[2], fc[2]);
          // W[t,u,v] = sum over aux terms sign coef R[t + tc, ...], pair index up to LAB + 1
          double W[ntuv(LAB + 1)];
#pragma unroll 1
          for (int N = 0; N <= LAB + 1; ++N)
#pragma unroll 1
            for (int t = N; t >= 0; --t)
#pragma unroll 1
              for (int u = N - t; u >= 0; --u) {
                const int v = N - t - u;
                double w = 0.0;
                for (int i0 = 0; i0 < n0; ++i0)
                  for (int i1 = 0; i1 < n1; ++i1)
                    for (int i2 = 0; i2 < n2; ++i2) {
                      const int ts = tc[0][i0] + tc[1][i1] + tc[2][i2];
                      const double c = fc[0][i0] * fc[1][i1] * fc[2][i2] * ((ts & 1) ? -1.0 : 1.0);
                      w = fma(c, R[tuv_idx(t + tc[0][i0], u + tc[1][i1], v + tc[2][i2])], w);
                    }
                W[tuv_idx(t, u, v)] = w;
              }
          const double wc = pt * comp_factor(LC, cc);
#pragma unroll 1
          for (int ca = 0; ca < NCA; ++ca)
#pragma unroll 1
            for (int cb = 0; cb < NCB; ++cb) {
              double wj = dP[cc] * sD[ca * NCB + cb];
              if (gP) wj = fma(kf, __ldg(gP + cc * nao2 + (long long)(mu0 + ca) * g.nao + nu0 + cb), wj);
              const double wt = wc * wj * comp_factor(LA, ca) * comp_factor(LB, cb);
              if (wt == 0.0) continue;
              const int ax[3] = {cart_x(LA, ca), cart_y(LA, ca), cart_z(LA, ca)};
              const int bx[3] = {cart_x(LB, cb), cart_y(LB, cb), cart_z(LB, cb)};
              double dA[3] = {0.0, 0.0, 0.0}, dC[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
              for (int t = 0; t <= ax[0] + bx[0] + 1; ++t)
#pragma unroll 1
                for (int u = 0; u <= ax[1] + bx[1] + 1; ++u)
#pragma unroll 1
                  for (int v = 0; v <= ax[2] + bx[2] + 1; ++v) {
                    const int tt[3] = {t, u, v};
                    // E factors per direction: plain E^{a b}, raised 2a E^{a+1 b} - a E^{a-1 b}
                    double e0[3], e1[3];
                    for (int q = 0; q < 3; ++q) {
                      const int i = ax[q], j = bx[q], k = tt[q];
                      e0[q] = (k <= i + j) ? sE[q][i][j][k] : 0.0;
                      double r = a2 * sE[q][i + 1][j][k];
                      if (i > 0 && k <= i - 1 + j) r -= i * sE[q][i - 1][j][k];
                      e1[q] = r;
                    }
                    if (t + u + v <= LAB + 1) {
                      const double w = W[tuv_idx(t, u, v)];
                      dA[0] = fma(e1[0] * e0[1] * e0[2], w, dA[0]);
                      dA[1] = fma(e0[0] * e1[1] * e0[2], w, dA[1]);
                      dA[2] = fma(e0[0] * e0[1] * e1[2], w, dA[2]);
                    }
                    // aux centre: the aux index shifted by one, with one more sign
                    const double e000 = e0[0] * e0[1] * e0[2];
                    if (e000 != 0.0 && t + u + v + 1 <= LAB + 1) {
                      dC[0] -= e000 * W[tuv_idx(t + 1, u, v)];
                      dC[1] -= e000 * W[tuv_idx(t, u + 1, v)];
                      dC[2] -= e000 * W[tuv_idx(t, u, v + 1)];
                    }
                  }
              for (int q = 0; q < 3; ++q) {
                gA[q] = fma(wt, dA[q], gA[q]);
                gCp[q] = fma(wt, dC[q], gCp[q]);
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

// Metric term: block per aux shell sp, threads over the aux shells sq on other
// atoms; adds -d_P d_Q d(P|Q)/dR_P (R_P moving alone) to the atom of sp.
__global__ void __launch_bounds__(128) grad2c_kernel(GradArgs g, AuxArgs aux, const int *aux_l, int nshell,
                                                     const double *__restrict__ boys_tab) {
  __shared__ double sRed[4][3];
  const int sp = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lp = aux_l[sp], np_ = (lp + 1) * (lp + 2) / 2;
  const int atom_p = g.aux_atom[sp];
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
  for (int sq = tid; sq < nshell; sq += blockDim.x) {
    if (g.aux_atom[sq] == atom_p) continue;
    const int lq = aux_l[sq], nq_ = (lq + 1) * (lq + 2) / 2;
    const double X = aux.center[3 * sp] - aux.center[3 * sq];
    const double Y = aux.center[3 * sp + 1] - aux.center[3 * sq + 1];
    const double Z = aux.center[3 * sp + 2] - aux.center[3 * sq + 2];
    const int L1 = lp + lq + 1;
#pragma unroll 1
    for (int kp = 0; kp < aux.nprim[sp]; ++kp)
#pragma unroll 1
      for (int kq = 0; kq < aux.nprim[sq]; ++kq) {
        const int ip0 = aux.prim_off[sp] + kp, iq0 = aux.prim_off[sq] + kq;
        const double a = aux.exps[ip0], gq = aux.exps[iq0];
        const double s = rsqrt(a + gq);
        const double al = a * gq * s * s;
        double F[9];
        boys_eval<5>(al * (X * X + Y * Y + Z * Z), boys_tab, F);  // lp + lq + 1 <= 5
        double R[ntuv(8)];
        hermite_R_rt<double>(L1, F, al, X, Y, Z, R);
        const double pref = 2.0 * 17.493418327624862846 * s * aux.cdiv[ip0] * aux.cdiv[iq0];
#pragma unroll 1
        for (int cp = 0; cp < np_; ++cp)
#pragma unroll 1
          for (int cq = 0; cq < nq_; ++cq) {
            const int P = aux.func_off[sp] + cp, Q = aux.func_off[sq] + cq;
            double wpq = g.cj * g.d[P] * g.d[Q];
            if (g.W) wpq = fma(g.ck, g.W[(long long)P * g.ldw + Q], wpq);
            const double w = pref * wpq * comp_factor(lp, cp) * comp_factor(lq, cq);
            int tp[3][2], tq[3][2], npp[3], nqq[3];
            double fp[3][2], fq[3][2];
            npp[0] = one_centre_terms(cart_x(lp, cp), aux.g1[ip0], tp[0], fp[0]);
            npp[1] = one_centre_terms(cart_y(lp, cp), aux.g1[ip0], tp[1], fp[1]);
            npp[2] = one_centre_terms(cart_z(lp, cp), aux.g1[ip0], tp[2], fp[2]);
            nqq[0] = one_centre_terms(cart_x(lq, cq), aux.g1[iq0], tq[0], fq[0]);
            nqq[1] = one_centre_terms(cart_y(lq, cq), aux.g1[iq0], tq[1], fq[1]);
            nqq[2] = one_centre_terms(cart_z(lq, cq), aux.g1[iq0], tq[2], fq[2]);
            double dx = 0.0, dy = 0.0, dz = 0.0;
            for (int i0 = 0; i0 < npp[0]; ++i0)
              for (int i1 = 0; i1 < npp[1]; ++i1)
                for (int i2 = 0; i2 < npp[2]; ++i2)
                  for (int j0 = 0; j0 < nqq[0]; ++j0)
                    for (int j1 = 0; j1 < nqq[1]; ++j1)
                      for (int j2 = 0; j2 < nqq[2]; ++j2) {
                        const int t = tp[0][i0] + tq[0][j0], u = tp[1][i1] + tq[1][j1], v = tp[2][i2] + tq[2][j2];
                        const double sg = ((tq[0][j0] + tq[1][j1] + tq[2][j2]) & 1) ? -1.0 : 1.0;
                        const double c = sg * fp[0][i0] * fp[1][i1] * fp[2][i2] * fq[0][j0] * fq[1][j1] * fq[2][j2];
                        // moving P: its Hermite index shifts by one (no extra sign)
                        dx = fma(c, R[tuv_idx(t + 1, u, v)], dx);
                        dy = fma(c, R[tuv_idx(t, u + 1, v)], dy);
                        dz = fma(c, R[tuv_idx(t, u, v + 1)], dz);
                      }
            acc[0] = fma(-w, dx, acc[0]);
            acc[1] = fma(-w, dy, acc[1]);
            acc[2] = fma(-w, dz, acc[2]);
          }
      }
  }
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (lane == 0)
    for (int q = 0; q < 3; ++q) sRed[warp][q] = acc[q];
  __syncthreads();
  if (tid < 3) atomicAdd(&g.grad[3 * atom_p + tid], sRed[0][tid] + sRed[1][tid] + sRed[2][tid] + sRed[3][tid]);
}

// Back substitution L^T d = r, one block: step i fixes d_i and removes it from
// the rows above (row i of L is contiguous, so the update is coalesced).
__global__ void __launch_bounds__(1024) lt_solve_kernel(const double *__restrict__ L, int n, int ld,
                                                        double *__restrict__ r, double *__restrict__ d) {
#pragma unroll 1
  for (int i = n - 1; i >= 0; --i) {
    __syncthreads();
    const double di = r[i] / L[(long long)i * ld + i];
    for (int j = threadIdx.x; j < i; j += blockDim.x) r[j] = fma(-L[(long long)i * ld + j], di, r[j]);
    if (threadIdx.x == 0) d[i] = di;
  }
}

void fitted_coefficients(const double *L, int n, int ld, const double *rho, double *work, double *d,
                         cudaStream_t st) {
  if (n == 0) return;
  DFJK_CUDA_CHECK(cudaMemcpyAsync(work, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  lt_solve_kernel<<<1, 1024, 0, st>>>(L, n, ld, work, d);
  DFJK_LAUNCHED();
}

void launch_grad3c(int la, int lb, int lc, const GradArgs &a, const OrbArgs &o, const AuxArgs &x,
                   const double *tab, cudaStream_t st) {
  if (a.npairs == 0 || a.naux_shells == 0) return;
  dim3 grid(ceil_div(a.npairs, a.pair_chunk), ceil_div(a.naux_shells, 128));
#define GRAD3C(LC_)                                                                            \
  DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, LC_><<<grid, 128, 0, st>>>(a, o, x, tab)))
  switch (lc) {
    case 0: GRAD3C(0); break;
    case 1: GRAD3C(1); break;
    case 2: GRAD3C(2); break;
    default: throw Error{DFJK_ERR_UNSUPPORTED, "aux class"};
  }
#undef GRAD3C
  DFJK_LAUNCHED();
}

void launch_grad2c(const GradArgs &a, const AuxArgs &x, const int *aux_l, int nshell, const double *tab,
                   cudaStream_t st) {
  if (nshell == 0) return;
  grad2c_kernel<<<nshell, 128, 0, st>>>(a, x, aux_l, nshell, tab);
  DFJK_LAUNCHED();
}

}  // namespace dfjk
