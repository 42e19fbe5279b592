// Mixed-precision path: not built yet; every entry reports DFJK_ERR_UNSUPPORTED.
#include "common.cuh"
#include "mixed.cuh"

namespace dfjk {

size_t mixed_B_bytes(int, int) { return 0; }
size_t mixed_B_resident_bytes(const MixedB &b) { return b.bytes; }
void mixed_alloc_B(MixedB &, int, int, cudaStream_t) {
  throw Error{DFJK_ERR_UNSUPPORTED, "mixed precision is not available in this build"};
}
void mixed_release_B(MixedB &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}
void mixed_release_work(MixedWork &w) {
  if (w.p) cudaFree(w.p);
  w.p = nullptr;
  w.bytes = 0;
}
void mixed_whiten_slab(MixedB &, const double *, int, int, const double *, const int *, const int *, int,
                       cudaStream_t) {
  throw Error{DFJK_ERR_UNSUPPORTED, "mixed precision is not available in this build"};
}
void mixed_build(MixedB &, MixedWork &, int, int, int, const double *, double *, double *, double *, double *,
                 double *, double *, int, cudaStream_t) {
  throw Error{DFJK_ERR_UNSUPPORTED, "mixed precision is not available in this build"};
}
void mixed_expand_B(const MixedB &, int, int, double *, cudaStream_t) {
  throw Error{DFJK_ERR_UNSUPPORTED, "mixed precision is not available in this build"};
}

}  // namespace dfjk
