// Point updates of the seven stencils (arXiv 1510.04995, Sect. 2.2, Listings 1-4, and the
// 27-point box operator and red-black Gauss-Seidel of Sect. 8.4) and the small
// device helpers the sweep kernels share.
//
// Every kernel of the library computes a lattice-site update (LUP) through exactly one of the
// functions below, with explicitly rounded operations (__f*_rn / __d*_rn / fma), so the naive
// sweep and the blocked sweep produce bit-identical grids: blocking only reorders independent
// updates (Sect. 2.1) and never changes a point's arithmetic.
//
// Term order follows the listings left to right; where the listing has "a*b + c" the product is
// fused into one fma (one rounding instead of two; the FP64 contract is 1e-12 normwise):
//   7pt const : acc = c0*V; acc += c1*(x+1 + x-1); acc += c1*(y+1 + y-1); acc += c1*(z+1 + z-1)
//   7pt var   : acc = C0*V; acc += C1*x+1; += C2*x-1; += C3*y+1; += C4*y-1; += C5*z+1; += C6*z-1
//   25pt const: lap = c0*V; for r=1..4: lap += c_r*(((((x+r + x-r) + y+r) + y-r) + z+r) + z-r)
//               U' = ((V + V) - U) + lap      (Listing 3 with the per-point factor equal to 1)
//   25pt var  : acc = C00*V; for r=1..4: acc += C(3r-2)*(x pair) + C(3r-1)*(y pair) + C(3r)*(z pair)
//               U' = ((V + V) - U) + acc
//   25pt Cgrid: lap as 25pt const; U' = fma(C, lap, (V + V) - U)   (Listing 3 as printed)
//   27pt box  : F, E, K = sums of the face, edge and corner neighbours, each taken over the
//               offsets in (dz, dy, dx) lexicographic order; acc = c0*V; acc += c1*F; += c2*E;
//               += c3*K
//   7pt RB-GS : the 7pt const formula for the points whose interior (x + y + z + t) is even at
//               time step (half-sweep) t; the others keep their value (the kernels select)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace girih {

// R: radius; NCOEF: coefficient grids; ORDER2: second order in time; BOX: diagonal neighbours
// (read through the accessor's b(dx, dy, dz)); RB: red-black colour mask on the update.
template <int S>
struct Traits;
template <>
struct Traits<0> { static constexpr int R = 1, NCOEF = 0; static constexpr bool ORDER2 = false, BOX = false, RB = false; };
template <>
struct Traits<1> { static constexpr int R = 1, NCOEF = 7; static constexpr bool ORDER2 = false, BOX = false, RB = false; };
template <>
struct Traits<2> { static constexpr int R = 4, NCOEF = 0; static constexpr bool ORDER2 = true, BOX = false, RB = false; };
template <>
struct Traits<3> { static constexpr int R = 4, NCOEF = 13; static constexpr bool ORDER2 = true, BOX = false, RB = false; };
template <>
struct Traits<4> { static constexpr int R = 4, NCOEF = 1; static constexpr bool ORDER2 = true, BOX = false, RB = false; };
template <>
struct Traits<5> { static constexpr int R = 1, NCOEF = 0; static constexpr bool ORDER2 = false, BOX = true, RB = false; };
template <>
struct Traits<6> { static constexpr int R = 1, NCOEF = 0; static constexpr bool ORDER2 = false, BOX = false, RB = true; };

template <typename T>
struct Ops;
template <>
struct Ops<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct Ops<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// Two FP32 values in one 64-bit register pair, operated on by the packed FP32 instructions
// (add/sub/mul/fma .rn.f32x2, sm_100 and later): each lane is rounded exactly as the scalar
// instruction would round it, so point_update<S, F2> gives, lane by lane, the bits of
// point_update<S, float> for two points, in half the FP instructions.
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 pack2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(F2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
template <>
struct Ops<F2> {
  static __device__ __forceinline__ F2 mul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ F2 add(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ F2 sub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
  }
  static __device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
  }
};

// An accessor A provides, for the point being updated:
//   A.c()       centre value of level t                 A.x(d), A.y(d), A.z(d)  neighbours at offset d
//   A.u()       centre value of level t-1 (ORDER2 only) A.k(g)                  coefficient grid g
//   A.b(dx, dy, dz)  neighbour at any offset in [-1, 1]^3 (BOX only)
template <int S, typename T, typename A>
__device__ __forceinline__ T point_update(const A& a, const T* cst) {
  using O = Ops<T>;
  if constexpr (S == 0 || S == 6) {
    const T c0 = cst[0], c1 = cst[1];
    T acc = O::mul(c0, a.c());
    acc = O::fma(c1, O::add(a.x(1), a.x(-1)), acc);
    acc = O::fma(c1, O::add(a.y(1), a.y(-1)), acc);
    acc = O::fma(c1, O::add(a.z(1), a.z(-1)), acc);
    return acc;
  } else if constexpr (S == 1) {
    T acc = O::mul(a.k(0), a.c());
    acc = O::fma(a.k(1), a.x(1), acc);
    acc = O::fma(a.k(2), a.x(-1), acc);
    acc = O::fma(a.k(3), a.y(1), acc);
    acc = O::fma(a.k(4), a.y(-1), acc);
    acc = O::fma(a.k(5), a.z(1), acc);
    acc = O::fma(a.k(6), a.z(-1), acc);
    return acc;
  } else if constexpr (S == 5) {
    T cls[4];
    bool first[4] = {true, true, true, true};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int m = (dx != 0) + (dy != 0) + (dz != 0);
          if (m == 0) continue;
          const T v = a.b(dx, dy, dz);
          cls[m] = first[m] ? v : O::add(cls[m], v);
          first[m] = false;
        }
    T acc = O::mul(cst[0], a.c());
    acc = O::fma(cst[1], cls[1], acc);
    acc = O::fma(cst[2], cls[2], acc);
    acc = O::fma(cst[3], cls[3], acc);
    return acc;
  } else if constexpr (S == 2 || S == 4) {
    const T v = a.c();
    T lap = O::mul(cst[0], v);
#pragma unroll
    for (int r = 1; r <= 4; ++r) {
      T s = O::add(a.x(r), a.x(-r));
      s = O::add(s, a.y(r));
      s = O::add(s, a.y(-r));
      s = O::add(s, a.z(r));
      s = O::add(s, a.z(-r));
      lap = O::fma(cst[r], s, lap);
    }
    if constexpr (S == 4) return O::fma(a.k(0), lap, O::sub(O::add(v, v), a.u()));
    return O::add(O::sub(O::add(v, v), a.u()), lap);
  } else {
    const T v = a.c();
    T acc = O::mul(a.k(0), v);
#pragma unroll
    for (int r = 1; r <= 4; ++r) {
      acc = O::fma(a.k(3 * r - 2), O::add(a.x(r), a.x(-r)), acc);
      acc = O::fma(a.k(3 * r - 1), O::add(a.y(r), a.y(-r)), acc);
      acc = O::fma(a.k(3 * r), O::add(a.z(r), a.z(-r)), acc);
    }
    return O::add(O::sub(O::add(v, v), a.u()), acc);
  }
}

// Arithmetic instructions per LUP of point_update (each intrinsic is one FP instruction):
// 7pt const 7, 7pt var 7, 25pt const 1 + 4*6 + 3 = 28, 25pt var 1 + 12*2 + 3 = 28, 25pt Cgrid
// 1 + 4*6 + 3 = 28.
// 27pt box 5 + 11 + 7 + 1 + 3 = 27; 7pt RB-GS 7 (computed for every point, kept for one colour).
__host__ __device__ constexpr int fp_instructions_per_lup(int s) {
  return (s < 2 || s == 6) ? 7 : (s == 5 ? 27 : 28);
}

// ---- small PTX helpers (sm_90+ cluster features, cp.async) -------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
// All threads of all blocks of the cluster; release/acquire orders shared::cluster stores.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cp_async(void* smem_dst, const float* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem_dst)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async(void* smem_dst, const double* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem_dst)), "l"(g) : "memory");
}
// 16-byte copy global -> shared through L2 only (cp.async.cg), completing with the thread's
// cp.async groups.  Both addresses must be 16-byte aligned.
__device__ __forceinline__ void cp_async16_cg(void* smem_dst, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16_cg_u32(uint32_t smem_dst, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_dst), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's committed cp.async groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace girih
