// Argument blocks and launchers of the integral kernels (integrals.cu).
#pragma once

#include <cuda_runtime.h>

namespace dfjk {

constexpr int REC_HDR = 5;  // p, Px, Py, Pz, c_a c_b K_ab 2 pi^(5/2)/p
int pair_record_len(int la, int lb);

struct OrbArgs {  // orbital shells, user order
  const double *center;  // 3 per shell
  const int *prim_off, *nprim;
  const double *exps, *coefs;  // coefs: normalised radial coefficients
  const int *func_off;         // first AO of the shell
};

struct AuxArgs {  // aux shells, internal order (sorted by l)
  const double *center;
  const int *prim_off, *nprim;
  const double *exps;
  const double *cdiv;  // normalised radial coefficient / exponent
  const double *g1;    // 1 / (2 exponent)
  const int *func_off; // first internal aux function of the shell
};

struct PairClassArgs {
  int npair;
  const int *shell_a, *shell_b;  // class-local arrays
  const long long *rec_off;      // record offset (doubles) of the pair
  double *rec;                   // all records
  double *q;                     // Schwarz factor per pair (class-local)
  const int *npp_of;             // primitive pairs per pair (class-local)
};

struct Eri3cArgs {
  const int *pairs;  // global ids of the kept pairs to process
  int npairs;
  const long long *rec_off;   // by global id
  const int *npp;             // primitive pairs, by global id
  const long long *pair_col;  // first column, by global id
  const double *rec;
  const int *aux_shells;  // internal aux shell ids of class lc
  int naux_shells;
  double *T;  // slab, [col - col_begin][ldT]
  long long col_begin;
  int ldT;
};

struct MetricArgs {
  int npair;
  const int *shell_p, *shell_q;
  double *V;
  int ldV;
};

struct OverlapArgs {
  int npair;
  const int *shell_a, *shell_b;
  double *S;
  int ldS;
};

void launch_pair_kernel(int la, int lb, const PairClassArgs &a, const OrbArgs &o, const double *tab,
                        cudaStream_t st);
// fp32: the diagonal (ab|ab) on the FP32 pipe (it only decides screening and
// the FP32 integral split, to about 1e-4 of its value).
void launch_schwarz(int la, int lb, const PairClassArgs &a, const double *tab, const float *tab32, bool fp32,
                    cudaStream_t st);
void launch_eri3c_l0(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st);
void launch_eri3c_l1(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st);
void launch_eri3c_l2(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st);
void launch_eri3c(int la, int lb, int lc, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                  cudaStream_t st);
// FP32 integrals of small shell pairs (same arguments, FP32 Boys table).
void launch_eri3c32_l0(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const float *tab, cudaStream_t st);
void launch_eri3c32_l1(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const float *tab, cudaStream_t st);
void launch_eri3c32_l2(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const float *tab, cudaStream_t st);
void launch_eri3c32(int la, int lb, int lc, const Eri3cArgs &a, const AuxArgs &x, const float *tab,
                    cudaStream_t st);
void launch_metric(int lp, int lq, const MetricArgs &a, const AuxArgs &x, const double *tab,
                   cudaStream_t st);
void launch_overlap(int la, int lb, const OverlapArgs &a, const OrbArgs &o, cudaStream_t st);
void launch_boys(int mmax, int n, const double *T, double *F, const double *tab, cudaStream_t st);

}  // namespace dfjk
