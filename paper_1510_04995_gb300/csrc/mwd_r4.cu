// Instantiations of the per-element wavefront-diamond kernel for the radius-4 stencils.
#include "mwd_kernel.cuh"

namespace girih {

template <int S, typename T>
static void* ptr_g(int G) {
  switch (G) {
    case 1: return (void*)&mwd_fed_kernel<S, T, 1>;
    case 2: return (void*)&mwd_fed_kernel<S, T, 2>;
    default: return (void*)&mwd_fed_kernel<S, T, 4>;
  }
}

void* mwd_kernel_r4(int stencil, int dtype, int G) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 2) return f64 ? ptr_g<2, double>(G) : ptr_g<2, float>(G);
  return f64 ? ptr_g<3, double>(G) : ptr_g<3, float>(G);
}

}  // namespace girih
