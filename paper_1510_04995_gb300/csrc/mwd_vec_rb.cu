// Instantiations of the aligned-layout wavefront-diamond kernel for red-black Gauss-Seidel on
// the 7-point operator (its blocked sweep runs on this path only).
#include "mwd_vec.cuh"

namespace girih {

template <typename T, bool TMA>
static void* vec_ptr_rb(int G) {
  switch (G) {
    case 1: return (void*)&mwd_vec_kernel<6, T, 1, TMA>;
    case 2: return (void*)&mwd_vec_kernel<6, T, 2, TMA>;
    default: return (void*)&mwd_vec_kernel<6, T, 4, TMA>;
  }
}

void* mwd_vec_kernel_rb(int dtype, int G, bool tma) {
  if (dtype == GIRIH_F64) return tma ? vec_ptr_rb<double, true>(G) : vec_ptr_rb<double, false>(G);
  return tma ? vec_ptr_rb<float, true>(G) : vec_ptr_rb<float, false>(G);
}

}  // namespace girih
