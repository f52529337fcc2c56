// Instantiations of the aligned-layout wavefront-diamond kernel for the 27-point box stencil
// (its blocked sweep runs on this path only).
#include "mwd_vec.cuh"

namespace girih {

template <typename T, bool TMA>
static void* vec_ptr_box(int G) {
  switch (G) {
    case 1: return (void*)&mwd_vec_kernel<5, T, 1, TMA>;
    case 2: return (void*)&mwd_vec_kernel<5, T, 2, TMA>;
    default: return (void*)&mwd_vec_kernel<5, T, 4, TMA>;
  }
}

void* mwd_vec_kernel_box(int dtype, int G, bool tma) {
  if (dtype == GIRIH_F64) return tma ? vec_ptr_box<double, true>(G) : vec_ptr_box<double, false>(G);
  return tma ? vec_ptr_box<float, true>(G) : vec_ptr_box<float, false>(G);
}

}  // namespace girih
