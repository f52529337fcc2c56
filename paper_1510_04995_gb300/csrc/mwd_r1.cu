// Instantiations of the wavefront-diamond kernel for the radius-1 (7-point) stencils.
#include "mwd_kernel.cuh"

namespace girih {

template <int S, typename T, bool B>
static void* ptr_g(int G) {
  switch (G) {
    case 1: return (void*)&mwd_fed_kernel<S, T, 1, B>;
    case 2: return (void*)&mwd_fed_kernel<S, T, 2, B>;
    case 4: return (void*)&mwd_fed_kernel<S, T, 4, B>;
    default: return (void*)&mwd_fed_kernel<S, T, 8, B>;
  }
}
template <int S, typename T>
static void* ptr_for(int G, bool bulk) {
  return bulk ? ptr_g<S, T, true>(G) : ptr_g<S, T, false>(G);
}

void* mwd_kernel_r1(int stencil, int dtype, int G, bool bulk) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 0) return f64 ? ptr_for<0, double>(G, bulk) : ptr_for<0, float>(G, bulk);
  return f64 ? ptr_for<1, double>(G, bulk) : ptr_for<1, float>(G, bulk);
}

}  // namespace girih
