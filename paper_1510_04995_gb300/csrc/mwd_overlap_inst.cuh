// Instantiations of the overlapped-slab persistent wavefront-diamond kernel (OVERLAP_PERSISTENT)
// for the radius-1 first-order stencils and the radius-4 ones, with GIRIH_OVL_ZS false (whole
// tiles, mwd_overlap.cu) or true (tiles split along z, mwd_overlap_zs.cu); the two translation
// units compile in parallel.
#pragma once
#include "mwd_overlap.cuh"

namespace girih {

template <int S, typename T>
static void* ovl_ptr(int G) {
  switch (G) {
    case 1: return (void*)&mwd_ovl_kernel<S, T, 1, GIRIH_OVL_ZS>;
    case 2: return (void*)&mwd_ovl_kernel<S, T, 2, GIRIH_OVL_ZS>;
    default: return (void*)&mwd_ovl_kernel<S, T, 4, GIRIH_OVL_ZS>;
  }
}

#if GIRIH_OVL_ZS
void* mwd_ovlz_kernel_ptr(int stencil, int dtype, int G) {
#else
void* mwd_ovlz_kernel_ptr(int stencil, int dtype, int G);
void* mwd_ovl_kernel_ptr(int stencil, int dtype, int G, bool zseg) {
  if (zseg) return mwd_ovlz_kernel_ptr(stencil, dtype, G);
#endif
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case GIRIH_7PT_CONST: return f64 ? ovl_ptr<0, double>(G) : ovl_ptr<0, float>(G);
    case GIRIH_7PT_VAR: return f64 ? ovl_ptr<1, double>(G) : ovl_ptr<1, float>(G);
    case GIRIH_7PT_RBGS: return f64 ? ovl_ptr<6, double>(G) : ovl_ptr<6, float>(G);
    case GIRIH_25PT_CONST: return f64 ? ovl_ptr<2, double>(G) : ovl_ptr<2, float>(G);
    case GIRIH_25PT_VAR: return f64 ? ovl_ptr<3, double>(G) : ovl_ptr<3, float>(G);
    case GIRIH_25PT_CGRID: return f64 ? ovl_ptr<4, double>(G) : ovl_ptr<4, float>(G);
    default: return nullptr;
  }
}

}  // namespace girih
