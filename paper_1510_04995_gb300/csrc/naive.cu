// Naive sweep (arXiv 1510.04995, Sect. 2.1.1): one full pass over the grid per time step.
//
// On the GPU this is the "optimal spatial blocking" reference of Sect. 5 (diamond width 0):
// every block owns a 32 x 16 tile of x-y columns over a chunk of z planes, each thread two
// columns (rows ty and ty+8).  Each thread keeps its columns' 2R+1 values along z in registers
// (rotated as the block walks up in z), the current z plane of the block (plus an R-wide halo)
// is staged in shared memory for the x and y neighbours (double-buffered, one barrier per plane),
// the columns' next planes are prefetched several iterations ahead into a register queue and the
// halo cells two planes ahead, so that enough loads are in flight to saturate HBM.  Offsets within
// a plane are 32-bit (a plane of the padded grid holds fewer than 2^31 elements).  Every input is read
// from HBM once per step (halo re-reads hit L2), every output written once: 2s bytes per LUP
// for the 7-point constant stencil, s = element size.
#include <algorithm>

#include "internal.h"
#include "stencil.cuh"

namespace girih {

template <int S, typename T>
struct NaiveAcc {
  const T* tc;       // centre of this thread's row in the shared tile
  int tw;            // tile row pitch
  const T* w;        // register window, w[R] = centre
  const T* coef;
  int64_t gs;        // grid stride
  int64_t p;         // padded linear index of the point
  T uc;              // level t-1 centre (second order)
  __device__ __forceinline__ T c() const { return w[Traits<S>::R]; }
  __device__ __forceinline__ T x(int d) const { return tc[d]; }
  __device__ __forceinline__ T y(int d) const { return tc[d * tw]; }
  __device__ __forceinline__ T z(int d) const { return w[Traits<S>::R + d]; }
  __device__ __forceinline__ T u() const { return uc; }
  __device__ __forceinline__ T k(int g) const { return __ldg(coef + g * gs + p); }
};

// Block = 32 x TY threads covering a 32 x (2*TY) tile of (x, y) columns over a chunk of z
// planes; each thread owns rows ty and ty + TY (two independent updates per plane).
template <int S, typename T, int TY, int PD>
__global__ void __launch_bounds__(32 * TY) naive_kernel(const NaiveArgs a) {
  constexpr int R = Traits<S>::R;
  constexpr int ROWS = 2 * TY;
  constexpr int TXW = 32 + 2 * R, TYW = ROWS + 2 * R;
  constexpr int NH = 2 * R * (32 + ROWS);                 // halo cells of the tile (star stencil)
  constexpr int HPT = (NH + 32 * TY - 1) / (32 * TY);     // halo cells per thread
  __shared__ T tile[2][TYW * TXW];                        // double-buffered: one barrier per plane
  const T* __restrict__ V = static_cast<const T*>(a.V);
  T* __restrict__ U = static_cast<T*>(a.U);
  const T* __restrict__ coef = static_cast<const T*>(a.coef);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = static_cast<T>(a.c[i]);

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = (int)a.g.nx, ny = (int)a.g.ny, nz = (int)a.g.nz;
  const int64_t plane = a.g.sy * a.g.ldx;
  const int ldx = (int)a.g.ldx;
  const int x = blockIdx.x * 32 + tx;
  const int z0 = blockIdx.z * a.zc;
  const int z1 = min(z0 + a.zc, nz);
  // the block starts at padded plane z0; all offsets below are relative to that plane
  const T* Vz = V + (int64_t)z0 * plane;
  T* Uz = U + (int64_t)(z0 + R) * plane;

  int yr[2];
  bool inb[2], act[2];
  int colo[2];  // offset of the column within a plane
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    yr[r] = blockIdx.y * ROWS + ty + r * TY;
    inb[r] = (x < nx + R) && (yr[r] < ny + R);
    act[r] = (x < nx) && (yr[r] < ny);
    colo[r] = (yr[r] + R) * ldx + (x + R);
  }

  // this thread's halo cells (fixed for the whole z walk): tile offset and plane offset
  int hoff[HPT], hcol[HPT];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int i = tid + k * 32 * TY;
    hoff[k] = -1;
    hcol[k] = -1;
    if (i < NH) {
      int hx, hy;
      if (i < 2 * R * 32) {
        const int r = i / 32;
        hx = R + (i % 32);
        hy = (r < R) ? r : ROWS + r;
      } else {
        const int j = i - 2 * R * 32, cc = j / ROWS;
        hy = R + j % ROWS;
        hx = (cc < R) ? cc : 32 + cc;
      }
      const int px = blockIdx.x * 32 + hx, py = blockIdx.y * ROWS + hy;
      hoff[k] = hy * TXW + hx;
      if (px < nx + 2 * R && py < ny + 2 * R) hcol[k] = py * ldx + px;
    }
  }

  // register windows (padded planes z..z+2R for interior plane z) and a queue of PD planes ahead
  T w[2][2 * R + 1], q[2][PD], hv[2][HPT];
  const int zlast = z1 - 1 + 2 * R - z0;  // last plane (relative) this block reads
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int i = 0; i <= 2 * R; ++i) w[r][i] = inb[r] ? Vz[i * plane + colo[r]] : T(0);
#pragma unroll
    for (int i = 0; i < PD; ++i)
      q[r][i] = (inb[r] && 2 * R + 1 + i <= zlast) ? Vz[(2 * R + 1 + i) * plane + colo[r]] : T(0);
  }
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    hv[0][k] = (hcol[k] >= 0) ? Vz[R * plane + hcol[k]] : T(0);
    hv[1][k] = (hcol[k] >= 0 && z0 + 1 < z1) ? Vz[(R + 1) * plane + hcol[k]] : T(0);
  }

  int buf = 0;
  for (int zr = 0; zr < z1 - z0; ++zr) {
    T* tl = tile[buf];
#pragma unroll
    for (int r = 0; r < 2; ++r) tl[(ty + r * TY + R) * TXW + tx + R] = w[r][R];
#pragma unroll
    for (int k = 0; k < HPT; ++k)
      if (hoff[k] >= 0) tl[hoff[k]] = hv[0][k];
    // halo cells two planes ahead
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
      hv[0][k] = hv[1][k];
      hv[1][k] = (hcol[k] >= 0 && z0 + zr + 2 < z1) ? Vz[(zr + 2 + R) * plane + hcol[k]] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (act[r]) {
        const int64_t off = (int64_t)zr * plane + colo[r];
        NaiveAcc<S, T> acc{tl + (ty + r * TY + R) * TXW + tx + R, TXW, w[r], coef, a.g.gstride,
                           (int64_t)(z0 + zr + R) * plane + colo[r], T(0)};
        if constexpr (Traits<S>::ORDER2) acc.uc = Uz[off];
        Uz[off] = point_update<S, T>(acc, cst);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) w[r][i] = w[r][i + 1];
      w[r][2 * R] = q[r][0];
#pragma unroll
      for (int i = 0; i < PD - 1; ++i) q[r][i] = q[r][i + 1];
      const int pz = zr + 2 * R + 1 + PD;
      q[r][PD - 1] = (inb[r] && pz <= zlast) ? Vz[pz * plane + colo[r]] : T(0);
    }
    buf ^= 1;
  }
}

constexpr int kTY = 8;

int naive_block_rows(int, int) { return 2 * kTY; }

template <int S, typename T>
static cudaError_t launch_one(const NaiveArgs& a, cudaStream_t st) {
  dim3 block(32, kTY);
  dim3 grid((unsigned)((a.g.nx + 31) / 32), (unsigned)((a.g.ny + 2 * kTY - 1) / (2 * kTY)),
            (unsigned)((a.g.nz + a.zc - 1) / a.zc));
  constexpr int PD = (Traits<S>::R == 4 && sizeof(T) == 8) ? 2 : 3;
  naive_kernel<S, T, kTY, PD><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_naive_step(int stencil, int dtype, const NaiveArgs& a, cudaStream_t st) {
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case 0: return f64 ? launch_one<0, double>(a, st) : launch_one<0, float>(a, st);
    case 1: return f64 ? launch_one<1, double>(a, st) : launch_one<1, float>(a, st);
    case 2: return f64 ? launch_one<2, double>(a, st) : launch_one<2, float>(a, st);
    default: return f64 ? launch_one<3, double>(a, st) : launch_one<3, float>(a, st);
  }
}

// Element-wise exchange of two equally sized arrays of W-byte words.
template <typename W>
__global__ void swap_kernel(W* a, W* b, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const W va = a[i], vb = b[i];
    a[i] = vb;
    b[i] = va;
  }
}

cudaError_t launch_swap(void* a, void* b, int64_t bytes, cudaStream_t st) {
  // girih_run guarantees 4-byte alignment and a byte count that is a multiple of 4; use 16-byte
  // words when both pointers and the size allow it (always the case for torch allocations).
  const uintptr_t al = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | (uintptr_t)bytes;
  if ((al & 15) == 0) {
    const int64_t n = bytes / 16;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (n > 0) swap_kernel<uint4><<<blocks, 256, 0, st>>>(static_cast<uint4*>(a), static_cast<uint4*>(b), n);
  } else {
    const int64_t n = bytes / 4;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (n > 0) swap_kernel<uint32_t><<<blocks, 256, 0, st>>>(static_cast<uint32_t*>(a), static_cast<uint32_t*>(b), n);
  }
  return cudaGetLastError();
}

}  // namespace girih
