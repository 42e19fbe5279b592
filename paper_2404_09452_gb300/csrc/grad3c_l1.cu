// Derivative 3-centre kernel instantiations for aux shells with l = 1 (split
// out so the translation units compile in parallel).
#include "grad3c.cuh"

namespace dfjk {

void launch_grad3c_l1(int la, int lb, const GradArgs &a, const OrbArgs &o, const AuxArgs &x, const double *tab,
                      cudaStream_t st) {
  dim3 grid(ceil_div(a.npairs, a.pair_chunk), ceil_div(a.naux_shells, 128));
  if (a.gam) {
    DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, 1, true><<<grid, 128, 0, st>>>(a, o, x, tab)));
  } else {
    DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, 1, false><<<grid, 128, 0, st>>>(a, o, x, tab)));
  }
}

}  // namespace dfjk
