// 3-centre kernel instantiations for aux shells with l = 0 (split out so the
// translation units compile in parallel).
#include "md.cuh"

namespace dfjk {

void launch_eri3c_l0(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st) {
  if (eri3c_use_coop_a(la, lb)) {  // (dd|s): the threads of an aux shell share R
    using Sh = CoopShapeA<2>;
    dim3 grid(a.npairs, ceil_div(a.naux_shells, Sh::NS));
    eri3c_coop_a_kernel<2, 2, double><<<grid, Sh::THREADS, 0, st>>>(a, x, tab);
    return;
  }
  dim3 grid(a.npairs, ceil_div(a.naux_shells, 128));
  DISPATCH_LALB(la, lb, (eri3c_kernel<A_, B_, 0><<<grid, 128, 0, st>>>(a, x, tab)));
}

}  // namespace dfjk
