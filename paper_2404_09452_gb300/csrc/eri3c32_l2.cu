// FP32 3-centre kernel instantiations for aux shells with l = 2 (small shell
// pairs; one translation unit per aux class so they compile in parallel).
#include "md.cuh"

namespace dfjk {

void launch_eri3c32_l2(int la, int lb, const Eri3cArgs &a, const AuxArgs &x, const float *tab,
                       cudaStream_t st) {
  if (eri3c_use_coop(la, lb, 2, true)) {  // the NCC threads of an aux shell share its work
    using Sh = CoopShape<2>;
    dim3 grid(a.npairs, ceil_div(a.naux_shells, Sh::NS));
    DISPATCH_LALB(la, lb, (eri3c_coop_kernel<A_, B_, 2, float><<<grid, Sh::THREADS, 0, st>>>(a, x, tab)));
    return;
  }
  dim3 grid(a.npairs, ceil_div(a.naux_shells, 128));
  DISPATCH_LALB(la, lb, (eri3c32_kernel<A_, B_, 2><<<grid, 128, 0, st>>>(a, x, tab)));
}

}  // namespace dfjk
