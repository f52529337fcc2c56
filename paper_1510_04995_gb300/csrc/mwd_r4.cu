// Instantiations of the wavefront-diamond kernel for the radius-4 (25-point) stencils.
#include "mwd_kernel.cuh"

namespace girih {

template <int S, typename T, bool B>
static void* ptr_g(int G) {  // radius-4 tiles use at most 4 pairs per thread
  return G == 1 ? (void*)&mwd_fed_kernel<S, T, 1, B> : (G == 2 ? (void*)&mwd_fed_kernel<S, T, 2, B> : (void*)&mwd_fed_kernel<S, T, 4, B>);
}
template <int S, typename T>
static void* ptr_for(int G, bool bulk) {
  return bulk ? ptr_g<S, T, true>(G) : ptr_g<S, T, false>(G);
}

void* mwd_kernel_r4(int stencil, int dtype, int G, bool bulk) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 2) return f64 ? ptr_for<2, double>(G, bulk) : ptr_for<2, float>(G, bulk);
  return f64 ? ptr_for<3, double>(G, bulk) : ptr_for<3, float>(G, bulk);
}

}  // namespace girih
