// Instantiations of the aligned-layout wavefront-diamond kernel for the radius-4 stencils.
#include "mwd_vec.cuh"

namespace girih {

template <int S, typename T, bool TMA>
static void* vec_ptr_t(int G) {
  switch (G) {
    case 1: return (void*)&mwd_vec_kernel<S, T, 1, TMA>;
    case 2: return (void*)&mwd_vec_kernel<S, T, 2, TMA>;
    default: return (void*)&mwd_vec_kernel<S, T, 4, TMA>;
  }
}

template <int S, typename T>
static void* vec_ptr(int G, bool tma) {
  return tma ? vec_ptr_t<S, T, true>(G) : vec_ptr_t<S, T, false>(G);
}

void* mwd_vec_kernel_r4(int stencil, int dtype, int G, bool tma) {
  const bool f64 = dtype == GIRIH_F64;
  if (stencil == 2) return f64 ? vec_ptr<2, double>(G, tma) : vec_ptr<2, float>(G, tma);
  return f64 ? vec_ptr<3, double>(G, tma) : vec_ptr<3, float>(G, tma);
}

}  // namespace girih
