// Gaussian integral kernels of the DF-J/K build, FP64, McMurchie-Davidson.
//
// Paper: Introduction, contribution 1 (density fitting evaluates 3-centre
// integrals on the GPU) and Sec. "Limitations and Future Development" (the
// integral scheme is an open choice; Rys quadrature was picked there for
// simplicity).  This file uses the McMurchie-Davidson scheme: the product of
// two Cartesian Gaussians is expanded in Hermite Gaussians at the product
// centre P,
//   x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = K_x sum_t E^{ij}_t Lambda_t(x; p, P_x),
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
//   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1},
// and Coulomb integrals between Hermite Gaussians reduce to
//   (Lambda_tuv(p,P) | Lambda_t'u'v'(q,Q)) = 2 pi^(5/2)/(p q sqrt(p+q))
//                                 (-1)^(t'+u'+v') R_{t+t',u+u',v+v'}(a, P-Q),
//   R^n_000 = (-2a)^n F_n(a |PQ|^2),  a = pq/(p+q),
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{tuv}  (same for u, v).
// A one-centre Gaussian x_C^k exp(-g x_C^2) has the Hermite expansion
// k=0: Lambda_0; k=1: Lambda_1/(2g); k=2: Lambda_0/(2g) + Lambda_2/(4g^2).
//
// FP64 is the scarce pipe on this GPU (about 1/62 of FP32), so the kernels are
// shaped to minimise FP64 instructions: pair quantities (p, P, K_ab and the
// products E^x E^y E^z for every term) are computed once per primitive pair by
// pair_kernel and broadcast from shared memory; index arithmetic, loads and
// register spills cost issue slots that the FP64 pipe leaves idle anyway.
#include <vector>

#include "md.cuh"

namespace dfjk {

int pair_record_len(int la, int lb) {
  static const int tab[3][3] = {{REC_HDR + nterms(0, 0), REC_HDR + nterms(0, 1), REC_HDR + nterms(0, 2)},
                                {REC_HDR + nterms(1, 0), REC_HDR + nterms(1, 1), REC_HDR + nterms(1, 2)},
                                {REC_HDR + nterms(2, 0), REC_HDR + nterms(2, 1), REC_HDR + nterms(2, 2)}};
  return tab[la][lb];
}

// ---- launchers ----------------------------------------------------------------

void launch_pair_kernel(int la, int lb, const PairClassArgs &a, const OrbArgs &o, const double *tab,
                        cudaStream_t st) {
  if (a.npair == 0) return;
  DISPATCH_LALB(la, lb, (pair_kernel<A_, B_><<<ceil_div(a.npair, 128), 128, 0, st>>>(a, o, tab)));
  DFJK_LAUNCHED();
}

void launch_schwarz(int la, int lb, const PairClassArgs &a, const double *tab, const float *tab32, bool fp32,
                    cudaStream_t st) {
  if (a.npair == 0) return;
  if (fp32) {
    DISPATCH_LALB(la, lb, (schwarz_kernel<A_, B_, float><<<a.npair, 64, 0, st>>>(a, tab32)));
  } else {
    DISPATCH_LALB(la, lb, (schwarz_kernel<A_, B_, double><<<a.npair, 64, 0, st>>>(a, tab)));
  }
  DFJK_LAUNCHED();
}

void launch_eri3c(int la, int lb, int lc, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                  cudaStream_t st) {
  if (a.npairs == 0 || a.naux_shells == 0) return;
  switch (lc) {
    case 0: launch_eri3c_l0(la, lb, a, x, tab, st); break;
    case 1: launch_eri3c_l1(la, lb, a, x, tab, st); break;
    case 2: launch_eri3c_l2(la, lb, a, x, tab, st); break;
    default: throw Error{DFJK_ERR_UNSUPPORTED, "aux class"};
  }
  DFJK_LAUNCHED();
}

void launch_eri3c32(int la, int lb, int lc, const Eri3cArgs &a, const AuxArgs &x, const float *tab,
                    cudaStream_t st) {
  if (a.npairs == 0 || a.naux_shells == 0) return;
  switch (lc) {
    case 0: launch_eri3c32_l0(la, lb, a, x, tab, st); break;
    case 1: launch_eri3c32_l1(la, lb, a, x, tab, st); break;
    case 2: launch_eri3c32_l2(la, lb, a, x, tab, st); break;
    default: throw Error{DFJK_ERR_UNSUPPORTED, "aux class"};
  }
  DFJK_LAUNCHED();
}

void launch_metric(int lp, int lq, const MetricArgs &a, const AuxArgs &x, const double *tab,
                   cudaStream_t st) {
  if (a.npair == 0) return;
  DISPATCH_LALB(lp, lq, (metric_kernel<A_, B_><<<ceil_div(a.npair, 128), 128, 0, st>>>(a, x, tab)));
  DFJK_LAUNCHED();
}

void launch_overlap(int la, int lb, const OverlapArgs &a, const OrbArgs &o, cudaStream_t st) {
  if (a.npair == 0) return;
  DISPATCH_LALB(la, lb, (overlap_kernel<A_, B_><<<ceil_div(a.npair, 128), 128, 0, st>>>(a, o)));
  DFJK_LAUNCHED();
}

void launch_boys(int mmax, int n, const double *T, double *F, const double *tab, cudaStream_t st) {
  if (n == 0) return;
  const int g = ceil_div(n, 128);
  switch (mmax) {
    case 0: boys_kernel<0><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 1: boys_kernel<1><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 2: boys_kernel<2><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 3: boys_kernel<3><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 4: boys_kernel<4><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 5: boys_kernel<5><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 6: boys_kernel<6><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 7: boys_kernel<7><<<g, 128, 0, st>>>(n, T, F, tab); break;
    case 8: boys_kernel<8><<<g, 128, 0, st>>>(n, T, F, tab); break;
    default: throw Error{DFJK_ERR_ARG, "mmax must be 0..8"};
  }
  DFJK_LAUNCHED();
}

// ---- Boys table (host) -----------------------------------------------------------

// F_m(T) = e^-T sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) in long double for
// the top order, then the downward recursion for the lower orders.
void boys_table_host(double *tab) {
  for (int k = 0; k < BOYS_NPT; ++k) {
    const long double T = (long double)k * (long double)BOYS_H;
    const int top = BOYS_NCOL - 1;
    long double term = 1.0L / (2 * top + 1), sum = term;
    for (int i = 1; i < 100000; ++i) {
      term *= 2.0L * T / (2 * top + 2 * i + 1);
      sum += term;
      if (term < 1e-22L * sum) break;
    }
    const long double e = expl(-T);
    long double f[BOYS_NCOL];
    f[top] = e * sum;
    for (int m = top - 1; m >= 0; --m) f[m] = (2.0L * T * f[m + 1] + e) / (2 * m + 1);
    for (int m = 0; m < BOYS_NCOL; ++m) tab[k * (BOYS_NCOL + 1) + m] = (double)f[m];
    tab[k * (BOYS_NCOL + 1) + BOYS_NCOL] = (double)e;
  }
}

}  // namespace dfjk
