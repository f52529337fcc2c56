// Naive sweep (arXiv 1510.04995, Sect. 2.1.1): one full pass over the grid per time step.
//
// On the GPU this is the "optimal spatial blocking" reference of Sect. 5 (diamond width 0):
// every block owns a 32 x ROWS column of x-y cells over a chunk of z planes.  Each thread keeps
// its column's 2R+1 values along z in registers (rotated as the block walks up in z), the current
// z plane of the block (plus an R-wide halo) is staged in shared memory for the x and y
// neighbours (double-buffered, one barrier per plane), and the column's next planes are
// prefetched several iterations ahead into a register queue so that enough loads are in flight.  Every input is read
// from HBM once per step (halo re-reads hit L2), every output written once: 2s bytes per LUP
// for the 7-point constant stencil, s = element size.
#include <algorithm>

#include "internal.h"
#include "stencil.cuh"

namespace girih {

template <int S, typename T, int ROWS>
struct NaiveAcc {
  T (*tile)[32 + 2 * Traits<S>::R];
  const T* w;        // register window, w[R] = centre
  const T* coef;
  int64_t gs, p;     // grid stride, padded linear index of the point
  int tx, ty;
  T uc;              // level t-1 centre (second order)
  __device__ __forceinline__ T c() const { return w[Traits<S>::R]; }
  __device__ __forceinline__ T x(int d) const { return tile[ty + Traits<S>::R][tx + Traits<S>::R + d]; }
  __device__ __forceinline__ T y(int d) const { return tile[ty + Traits<S>::R + d][tx + Traits<S>::R]; }
  __device__ __forceinline__ T z(int d) const { return w[Traits<S>::R + d]; }
  __device__ __forceinline__ T u() const { return uc; }
  __device__ __forceinline__ T k(int g) const { return __ldg(coef + g * gs + p); }
};

template <int S, typename T, int ROWS, int PD>
__global__ void __launch_bounds__(32 * ROWS) naive_kernel(const NaiveArgs a) {
  constexpr int R = Traits<S>::R;
  constexpr int TXW = 32 + 2 * R, TYW = ROWS + 2 * R;
  constexpr int NH = 2 * R * (32 + ROWS);                 // halo cells of the tile (star stencil)
  constexpr int HPT = (NH + 32 * ROWS - 1) / (32 * ROWS);  // halo cells per thread
  __shared__ T tile[2][TYW][TXW];                           // double-buffered: one barrier per plane
  const T* __restrict__ V = static_cast<const T*>(a.V);
  T* __restrict__ U = static_cast<T*>(a.U);
  const T* __restrict__ coef = static_cast<const T*>(a.coef);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = static_cast<T>(a.c[i]);

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int64_t nx = a.g.nx, ny = a.g.ny, nz = a.g.nz, ldx = a.g.ldx, sy = a.g.sy;
  const int64_t plane = sy * ldx;
  const int64_t x = (int64_t)blockIdx.x * 32 + tx, y = (int64_t)blockIdx.y * ROWS + ty;
  const bool inb = (x < nx + R) && (y < ny + R);  // this thread's cell exists in the padded grid
  const bool active = (x < nx) && (y < ny);
  const int64_t z0 = (int64_t)blockIdx.z * a.zc;
  const int64_t z1 = min(z0 + (int64_t)a.zc, nz);
  const int64_t col = (y + R) * ldx + (x + R);  // offset of this column within a plane
  const int64_t zlast = z1 - 1 + 2 * R;         // last padded plane this block reads

  // this thread's halo cells (fixed for the whole z walk)
  int hoff[HPT];
  int64_t hcol[HPT];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int i = tid + k * 32 * ROWS;
    int hx = 0, hy = 0;
    bool ok = i < NH;
    if (ok) {
      if (i < 2 * R * 32) {
        const int r = i / 32;
        hx = R + (i % 32);
        hy = (r < R) ? r : ROWS + r;
      } else {
        const int j = i - 2 * R * 32, cc = j / ROWS;
        hy = R + j % ROWS;
        hx = (cc < R) ? cc : 32 + cc;
      }
      const int64_t px = (int64_t)blockIdx.x * 32 + hx, py = (int64_t)blockIdx.y * ROWS + hy;
      ok = px < nx + 2 * R && py < ny + 2 * R;
      hcol[k] = ok ? py * ldx + px : -1;
    } else {
      hcol[k] = -1;
    }
    hoff[k] = (i < NH) ? hy * TXW + hx : -1;
  }

  // register window w (padded planes z..z+2R for interior plane z) and a queue of PD planes ahead:
  // PD outstanding loads per thread keep enough bytes in flight to saturate HBM.
  T w[2 * R + 1], q[PD], hv[HPT];
#pragma unroll
  for (int i = 0; i <= 2 * R; ++i) w[i] = inb ? V[(z0 + i) * plane + col] : T(0);
#pragma unroll
  for (int i = 0; i < PD; ++i) {
    const int64_t pz = z0 + 2 * R + 1 + i;
    q[i] = (inb && pz <= zlast) ? V[pz * plane + col] : T(0);
  }
#pragma unroll
  for (int k = 0; k < HPT; ++k) hv[k] = (hcol[k] >= 0) ? V[(z0 + R) * plane + hcol[k]] : T(0);

  int buf = 0;
  for (int64_t z = z0; z < z1; ++z) {
    T(*tl)[TXW] = tile[buf];
    tl[ty + R][tx + R] = w[R];
#pragma unroll
    for (int k = 0; k < HPT; ++k)
      if (hoff[k] >= 0) (&tl[0][0])[hoff[k]] = hv[k];
    // prefetch the next plane's halo cells
#pragma unroll
    for (int k = 0; k < HPT; ++k) hv[k] = (hcol[k] >= 0 && z + 1 < z1) ? V[(z + 1 + R) * plane + hcol[k]] : T(0);
    __syncthreads();
    if (active) {
      const int64_t p = (z + R) * plane + col;
      NaiveAcc<S, T, ROWS> acc{tl, w, coef, a.g.gstride, p, tx, ty, T(0)};
      if constexpr (Traits<S>::ORDER2) acc.uc = U[p];
      U[p] = point_update<S, T>(acc, cst);
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) w[i] = w[i + 1];
    w[2 * R] = q[0];
#pragma unroll
    for (int i = 0; i < PD - 1; ++i) q[i] = q[i + 1];
    {
      const int64_t pz = z + 2 * R + 1 + PD;
      q[PD - 1] = (inb && pz <= zlast) ? V[pz * plane + col] : T(0);
    }
    buf ^= 1;
  }
}

constexpr int kRows = 8;

int naive_block_rows(int, int) { return kRows; }

template <int S, typename T>
static cudaError_t launch_one(const NaiveArgs& a, cudaStream_t st) {
  dim3 block(32, kRows);
  dim3 grid((unsigned)((a.g.nx + 31) / 32), (unsigned)((a.g.ny + kRows - 1) / kRows),
            (unsigned)((a.g.nz + a.zc - 1) / a.zc));
  naive_kernel<S, T, kRows, (sizeof(T) == 8 ? 3 : 4)><<<grid, block, 0, st>>>(a);
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
