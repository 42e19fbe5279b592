// Nuclear gradient of the density-fitted Coulomb energy (grad.cu).
#pragma once

#include <cuda_runtime.h>

#include "integrals.cuh"

namespace dfjk {

struct GradArgs {
  const int *pairs;  // global ids of the kept pairs of one class
  int npairs;
  const int *pair_a, *pair_b;  // shells of a pair, by global id
  int pair_chunk;              // pairs per block
  const int *aux_shells;       // aux shell ids of one class
  int naux_shells;
  const double *d;  // fitted coefficients V^-1 u, one per aux function
  const double *D;  // density, nao x nao row-major
  int nao;
  double cj;  // weight of the Coulomb term: 3c weights cj d_P D_mu nu, 2c cj d_P d_Q
  // exchange term (gam == nullptr: none): 3c weights ck Gam[P][mu][nu],
  // 2c weights ck W[P][ldw]
  const double *gam, *W;
  int ldw;
  double ck;
  const int *orb_atom, *aux_atom;  // atom of each shell
  double *grad;                    // natom x 3, accumulated with atomicAdd
};

// d = L^-T rho = (L^-1)^T rho from the resident inverse (row-major, ld); work
// holds 16 n doubles.
void fitted_coefficients(const double *Linv, int n, int ld, const double *rho, double *work, double *d,
                         cudaStream_t st);
// sum_P sum_{mu nu} Gam_P,mu nu d(P|mu nu)/dR for pair class (la, lb), aux
// class lc, Gam = cj d_P D_mu nu + ck gam[P][mu][nu].
// f32: Coulomb-only weights evaluated in FP32 (pairs below the FP32 threshold).
void launch_grad3c(int la, int lb, int lc, const GradArgs &a, const OrbArgs &o, const AuxArgs &x,
                   const double *tab, const float *tab32, bool f32, cudaStream_t st);
void launch_grad3c_l0(int la, int lb, const GradArgs &a, const OrbArgs &o, const AuxArgs &x, const double *tab,
                      const float *tab32, bool f32, cudaStream_t st);
void launch_grad3c_l1(int la, int lb, const GradArgs &a, const OrbArgs &o, const AuxArgs &x, const double *tab,
                      const float *tab32, bool f32, cudaStream_t st);
void launch_grad3c_l2(int la, int lb, const GradArgs &a, const OrbArgs &o, const AuxArgs &x, const double *tab,
                      const float *tab32, bool f32, cudaStream_t st);
// -sum_PQ Wt_PQ dV_PQ/dR / 2 over all aux shells, Wt = cj d d^T + ck W
// (aux_l: l of each shell).
void launch_grad2c(const GradArgs &a, const AuxArgs &x, const int *aux_l, int nshell, const double *tab,
                   cudaStream_t st);

}  // namespace dfjk
