// Instantiations of the wavefront-diamond kernel for the radius-1 (7-point) stencils.
#include "mwd_kernel.cuh"

namespace girih {

template <int S, typename T>
static void* ptr_for(int G, bool bulk) {
  if (bulk) return G == 1 ? (void*)&mwd_fed_kernel<S, T, 1, true> : (G == 2 ? (void*)&mwd_fed_kernel<S, T, 2, true> : (void*)&mwd_fed_kernel<S, T, 4, true>);
  return G == 1 ? (void*)&mwd_fed_kernel<S, T, 1, false> : (G == 2 ? (void*)&mwd_fed_kernel<S, T, 2, false> : (void*)&mwd_fed_kernel<S, T, 4, false>);
}

void* mwd_kernel_r1(int stencil, int dtype, int G, bool bulk) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 0) return f64 ? ptr_for<0, double>(G, bulk) : ptr_for<0, float>(G, bulk);
  return f64 ? ptr_for<1, double>(G, bulk) : ptr_for<1, float>(G, bulk);
}

}  // namespace girih
