// 3-centre kernel instantiations for aux shells with l = 2 (split out so the
// translation units compile in parallel).
#include "md.cuh"

namespace dfjk {

void launch_eri3c_l2(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st) {
  // aux shells of the class split evenly into blocks of at most 128 threads
  const int nblk = ceil_div(a.naux_shells, 128);
  const int bs = ((ceil_div(a.naux_shells, nblk) + 31) / 32) * 32;
  dim3 grid(a.npairs, nblk);
  DISPATCH_LALB(la, lb, (eri3c_kernel<A_, B_, 2><<<grid, bs, 0, st>>>(a, x, tab)));
}

}  // namespace dfjk
