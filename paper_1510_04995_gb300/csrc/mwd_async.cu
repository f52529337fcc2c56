// Instantiations of the neighbour-synchronised persistent wavefront-diamond kernel
// (RELAXED_PERSISTENT) for the radius-1 first-order stencils.
#include "mwd_async.cuh"

namespace girih {

template <int S, typename T>
static void* async_ptr(int G) {
  switch (G) {
    case 1: return (void*)&mwd_async_kernel<S, T, 1>;
    case 2: return (void*)&mwd_async_kernel<S, T, 2>;
    default: return (void*)&mwd_async_kernel<S, T, 4>;
  }
}

void* mwd_async_kernel_ptr(int stencil, int dtype, int G) {
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case GIRIH_7PT_CONST: return f64 ? async_ptr<0, double>(G) : async_ptr<0, float>(G);
    case GIRIH_7PT_VAR: return f64 ? async_ptr<1, double>(G) : async_ptr<1, float>(G);
    case GIRIH_7PT_RBGS: return f64 ? async_ptr<6, double>(G) : async_ptr<6, float>(G);
    default: return nullptr;
  }
}

}  // namespace girih
