// Mixed-precision representation of B and the tensor-core J/K path (mixed.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace dfjk {

struct MixedB {
  void *p = nullptr;
  size_t bytes = 0;
};
struct MixedWork {
  void *p = nullptr;
  size_t bytes = 0;
};

size_t mixed_B_bytes(int nao, int naux_pad);
size_t mixed_B_resident_bytes(const MixedB &b);
void mixed_alloc_B(MixedB &b, int nao, int naux_pad, cudaStream_t st);
void mixed_release_B(MixedB &b);
void mixed_release_work(MixedWork &w);
void mixed_whiten_slab(MixedB &b, const double *T, int ncols, int np, const double *Linv,
                       const int *colmu, const int *colnu, int nao, cudaStream_t st);
void mixed_build(MixedB &b, MixedWork &w, int nao, int np, int nocc, const double *C, double *D,
                 double *rho, double *rho_work, double *J, double *K, double *Kpart, int ksplit,
                 cudaStream_t st);
void mixed_expand_B(const MixedB &b, int nao, int np, double *out, cudaStream_t st);

}  // namespace dfjk
