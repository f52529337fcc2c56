// Instantiations of the aligned-layout wavefront-diamond kernel for the 25-point stencil with
// the per-point factor grid (Listing 3 as printed); a translation unit of its own so that the
// radius-4 instantiations compile in parallel.
#include "mwd_vec.cuh"

namespace girih {

template <typename T, bool TMA>
static void* vec_ptr_cg(int G) {
  switch (G) {
    case 1: return (void*)&mwd_vec_kernel<4, T, 1, TMA>;
    case 2: return (void*)&mwd_vec_kernel<4, T, 2, TMA>;
    default: return (void*)&mwd_vec_kernel<4, T, 4, TMA>;
  }
}

void* mwd_vec_kernel_cg(int dtype, int G, bool tma) {
  if (dtype == GIRIH_F64) return tma ? vec_ptr_cg<double, true>(G) : vec_ptr_cg<double, false>(G);
  return tma ? vec_ptr_cg<float, true>(G) : vec_ptr_cg<float, false>(G);
}

}  // namespace girih
