// Nuclear gradient of the density-fitted Coulomb and exchange energies (FP64).
//
// Both energies have the form E = sum_PQ (V^-1)_PQ M_PQ / 2, with M_PQ = u_P u_Q,
// u_P = sum_{mu nu} (P|mu nu) D_mu nu (E_J) or M_PQ = Tr(D T_P D T_Q) (E_K), so
// at fixed D
//   dE/dR = sum_P sum_{mu nu} G_P,mu nu d(P|mu nu)/dR - sum_PQ W_PQ dV_PQ/dR / 2
// with G_P = d_P D, W = d d^T, d = V^-1 u = L^-T rho for E_J (rho = B vec D,
// the build's fitted vector), and G_P = C Z_P C^T, W = Z Z^T,
// Z_P = sum_Q (L^-1)_QP C^T B_Q C for E_K (formed by the host code with GEMMs).
// Derivatives of the integrals, McMurchie-Davidson form:
//  * orbital centre A:  d/dA_x [x_A^i e^{-a x_A^2}] = 2a x_A^{i+1} e - i x_A^{i-1} e,
//    i.e. the E^{i+1, j} and E^{i-1, j} Hermite coefficients of the pair;
//  * one-centre (aux) Gaussian at C: d/dC_x Lambda_t = Lambda_{t+1}, a shift of
//    the Hermite index;
//  * the second orbital centre B by translational invariance, dB = -(dA + dC),
//    triple by triple.
// For the metric term only pairs on different atoms contribute (the
// derivatives of same-atom pairs cancel), each as -W_PQ d(P|Q)/dR_P on the atom
// of P.  This file: the fitted coefficients, the metric term and the
// launchers; the 3-centre derivative kernel is in grad3c.cuh.
#include "grad.cuh"
#include "md.cuh"

namespace dfjk {

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

// d[Q] = sum_{P >= Q} Linv[P][Q] rho[P] (Linv = L^-1, lower triangular, row
// P contiguous): a thread per Q, the P range split over blockIdx.y into
// partial sums that a second kernel adds in a fixed order (deterministic).
constexpr int LT_SPLIT = 16;
__global__ void linv_t_partial_kernel(const double *__restrict__ Linv, int n, int ld,
                                      const double *__restrict__ rho, double *__restrict__ part) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int len = (n + LT_SPLIT - 1) / LT_SPLIT, p0 = blockIdx.y * len, p1 = min(n, p0 + len);
  double s = 0.0;
  if (q < n)
    for (int p = max(p0, q); p < p1; ++p) s = fma(Linv[(long long)p * ld + q], rho[p], s);
  if (q < n) part[(long long)blockIdx.y * n + q] = s;
}

__global__ void linv_t_sum_kernel(const double *__restrict__ part, int n, double *__restrict__ d) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double s = 0.0;
  for (int k = 0; k < LT_SPLIT; ++k) s += part[(long long)k * n + q];
  d[q] = s;
}

void fitted_coefficients(const double *Linv, int n, int ld, const double *rho, double *work, double *d,
                         cudaStream_t st) {
  if (n == 0) return;
  linv_t_partial_kernel<<<dim3(ceil_div(n, 128), LT_SPLIT), 128, 0, st>>>(Linv, n, ld, rho, work);
  DFJK_LAUNCHED();
  linv_t_sum_kernel<<<ceil_div(n, 128), 128, 0, st>>>(work, n, d);
  DFJK_LAUNCHED();
}

void launch_grad3c(int la, int lb, int lc, const GradArgs &a, const OrbArgs &o, const AuxArgs &x,
                   const double *tab, const float *tab32, bool f32, cudaStream_t st) {
  if (a.npairs == 0 || a.naux_shells == 0) return;
  if (f32 && a.gam) throw Error{DFJK_ERR_UNSUPPORTED, "FP32 gradient weights are Coulomb-only"};
  switch (lc) {
    case 0: launch_grad3c_l0(la, lb, a, o, x, tab, tab32, f32, st); break;
    case 1: launch_grad3c_l1(la, lb, a, o, x, tab, tab32, f32, st); break;
    case 2: launch_grad3c_l2(la, lb, a, o, x, tab, tab32, f32, st); break;
    default: throw Error{DFJK_ERR_UNSUPPORTED, "aux class"};
  }
  DFJK_LAUNCHED();
}

void launch_grad2c(const GradArgs &a, const AuxArgs &x, const int *aux_l, int nshell, const double *tab,
                   cudaStream_t st) {
  if (nshell == 0) return;
  grad2c_kernel<<<nshell, 128, 0, st>>>(a, x, aux_l, nshell, tab);
  DFJK_LAUNCHED();
}

}  // namespace dfjk
