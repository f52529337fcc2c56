// Instantiations of the per-element wavefront-diamond kernel for the 25-point stencil with the
// per-point factor grid (Listing 3 as printed).
#include "mwd_kernel.cuh"

namespace girih {

template <typename T>
static void* ptr_cg(int G) {
  switch (G) {
    case 1: return (void*)&mwd_fed_kernel<4, T, 1>;
    case 2: return (void*)&mwd_fed_kernel<4, T, 2>;
    default: return (void*)&mwd_fed_kernel<4, T, 4>;
  }
}

void* mwd_kernel_cg(int dtype, int G) { return dtype == GIRIH_F64 ? ptr_cg<double>(G) : ptr_cg<float>(G); }

}  // namespace girih
