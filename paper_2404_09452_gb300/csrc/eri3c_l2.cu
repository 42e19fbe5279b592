// 3-centre kernel instantiations for aux shells with l = 2 (split out so the
// translation units compile in parallel).
#include "md.cuh"

namespace dfjk {

void launch_eri3c_l2(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const double *tab,
                     cudaStream_t st) {
  if (eri3c_use_coop(la, lb, 2, false)) {  // the NCC threads of an aux shell share its work
    using Sh = CoopShape<2>;
    dim3 grid(a.npairs, ceil_div(a.naux_shells, Sh::NS));
    DISPATCH_LALB(la, lb, (eri3c_coop_kernel<A_, B_, 2, double><<<grid, Sh::THREADS, 0, st>>>(a, x, tab)));
    return;
  }
  dim3 grid(a.npairs, ceil_div(a.naux_shells, 128));
  DISPATCH_LALB(la, lb, (eri3c_kernel<A_, B_, 2><<<grid, 128, 0, st>>>(a, x, tab)));
}

}  // namespace dfjk
