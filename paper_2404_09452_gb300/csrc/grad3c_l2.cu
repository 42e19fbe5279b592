// Derivative 3-centre kernel instantiations for aux shells with l = 2 (split
// out so the translation units compile in parallel).
#include "grad3c.cuh"

namespace dfjk {

void launch_grad3c_l2(int la, int lb, const GradArgs &a, const OrbArgs &o, const AuxArgs &x, const double *tab,
                      const float *tab32, bool f32, cudaStream_t st) {
  dim3 grid(ceil_div(a.npairs, a.pair_chunk), ceil_div(a.naux_shells, 128));
  if (a.gam) {
    DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, 2, true, false><<<grid, 128, 0, st>>>(a, o, x, tab, tab32)));
  } else if (f32) {
    DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, 2, false, true><<<grid, 128, 0, st>>>(a, o, x, tab, tab32)));
  } else {
    DISPATCH_LALB(la, lb, (grad3c_kernel<A_, B_, 2, false, false><<<grid, 128, 0, st>>>(a, o, x, tab, tab32)));
  }
}

}  // namespace dfjk
