// Instantiations of the per-element wavefront-diamond kernel for the radius-1 stencils.
#include "mwd_kernel.cuh"

namespace girih {

template <int S, typename T>
static void* ptr_g(int G) {
  switch (G) {
    case 1: return (void*)&mwd_fed_kernel<S, T, 1>;
    case 2: return (void*)&mwd_fed_kernel<S, T, 2>;
    case 4: return (void*)&mwd_fed_kernel<S, T, 4>;
    default: return (void*)&mwd_fed_kernel<S, T, 8>;
  }
}

void* mwd_kernel_r1(int stencil, int dtype, int G) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 0) return f64 ? ptr_g<0, double>(G) : ptr_g<0, float>(G);
  return f64 ? ptr_g<1, double>(G) : ptr_g<1, float>(G);
}

}  // namespace girih
