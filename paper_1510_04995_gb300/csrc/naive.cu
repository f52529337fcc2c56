// Naive sweep (arXiv 1510.04995, Sect. 2.1.1): one full pass over the grid per time step.
//
// On the GPU this is the "optimal spatial blocking" reference of Sect. 5 (diamond width 0):
// every block owns a (32*VX) x 2TY tile of x-y columns over a chunk of z planes, each thread two
// rows (ty and ty+TY) of VX columns.  The tile's planes (with their R-wide halo) are staged into a
// shared-memory ring by cp.async several planes ahead of use; each thread keeps its columns'
// 2R+1 values along z in registers (rotated as the block walks up in z).  Every input is read
// from HBM once per step (halo re-reads hit L2), every output written once: 2s bytes per LUP
// for the 7-point constant stencil, s = element size.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "stencil.cuh"

namespace girih {

template <int S, typename T, int TW>
struct NaiveAcc {  // one column of the thread's VX columns
  const T* tc;       // centre of this thread's cell in the shared plane tile (row stride TW)
  const T* w;        // register window, w[R] = centre
  const T* kv;       // coefficient values of this point (variable stencils)
  T uc;              // level t-1 centre (second order)
  const T* tcm;      // box stencil: the same cell in the planes below and above
  const T* tcp;
  __device__ __forceinline__ T c() const { return w[Traits<S>::R]; }
  __device__ __forceinline__ T x(int d) const { return tc[d]; }
  __device__ __forceinline__ T y(int d) const { return tc[d * TW]; }
  __device__ __forceinline__ T z(int d) const { return w[Traits<S>::R + d]; }
  __device__ __forceinline__ T u() const { return uc; }
  __device__ __forceinline__ T k(int g) const { return kv[g]; }
  __device__ __forceinline__ T b(int dx, int dy, int dz) const {
    if (dx == 0 && dy == 0) return w[Traits<S>::R + dz];
    return (dz < 0 ? tcm : (dz > 0 ? tcp : tc))[dy * TW + dx];
  }
};

// Two columns of the thread as one packed accessor: every value is the pair of the two columns'
// values (FP32 sweeps with an even number of columns per thread).  D: the second column's offset
// from the first, 32 (radius 1: the interior starts at an odd shared column, so pairs of
// neighbours are packed from single loads) or 1 (radius 4: the first column is even, so pairs of
// y neighbours and of even x offsets are single 8-byte shared loads, and the odd x offsets are
// assembled from the halves of the even ones).
template <int S, int TW, int D>
struct NaiveAcc2 {
  const float* tc;  // first column's cell in the shared plane tile
  const float* w0;  // the two columns' register windows
  const float* w1;
  const float* kv0;
  const float* kv1;
  F2 uc;
  const float* tcm;
  const float* tcp;
  __device__ __forceinline__ F2 c() const { return pack2(w0[Traits<S>::R], w1[Traits<S>::R]); }
  __device__ __forceinline__ F2 ld2(int o) const {  // the pair at tc + o (D = 1: o even)
    if constexpr (D == 1) return F2{*reinterpret_cast<const unsigned long long*>(tc + o)};
    return pack2(tc[o], tc[o + D]);
  }
  __device__ __forceinline__ F2 x(int d) const {
    if constexpr (D == 1) {
      if (d & 1) {  // (c+d, c+d+1): the high half of the pair at d-1, the low half of the pair at d+1
        float a0, a1, b0, b1;
        unpack2(d - 1 == 0 ? c() : ld2(d - 1), a0, a1);
        unpack2(d + 1 == 0 ? c() : ld2(d + 1), b0, b1);
        return pack2(a1, b0);
      }
    }
    return ld2(d);
  }
  __device__ __forceinline__ F2 y(int d) const { return ld2(d * TW); }
  __device__ __forceinline__ F2 z(int d) const { return pack2(w0[Traits<S>::R + d], w1[Traits<S>::R + d]); }
  __device__ __forceinline__ F2 u() const { return uc; }
  __device__ __forceinline__ F2 k(int g) const { return pack2(kv0[g], kv1[g]); }
  __device__ __forceinline__ F2 b(int dx, int dy, int dz) const {
    if (dx == 0 && dy == 0) return z(dz);
    const float* q = (dz < 0 ? tcm : (dz > 0 ? tcp : tc)) + dy * TW + dx;
    return pack2(q[0], q[D]);
  }
};

// The 27-point box stencil's packed 2x2 block (FP32, two columns per thread): q[row][plane][dx]
// holds, for rows y0-1 .. y0+2 and planes z-1 .. z+1 of the thread's rows y0, y0+1 and columns
// c, c+1, the pairs of columns (c-1, c), (c, c+1), (c+1, c+2); row ROW of the block reads its
// 26 neighbours and centre from them.
template <int ROW>
struct BoxAcc2 {
  const F2 (*q)[3][3];
  __device__ __forceinline__ F2 c() const { return q[ROW + 1][1][1]; }
  __device__ __forceinline__ F2 z(int d) const { return q[ROW + 1][1 + d][1]; }
  __device__ __forceinline__ F2 b(int dx, int dy, int dz) const { return q[ROW + 1 + dy][1 + dz][1 + dx]; }
};

// Block = 32 x TY threads over a 32 x 2TY tile of (x, y) columns and a chunk of z planes; each
// thread owns rows ty and ty + TY.  The tile's planes (with the R-wide halo) stream through a
// ring of NP = R + PD + 2 (+1 for the box stencil) shared-memory slots filled PD planes ahead of
// use (one commit group per plane): at the update of plane z the ring holds padded planes z+R
// (the x/y neighbours; from z+R-1 for the box stencil, whose diagonal neighbours also lie in the
// planes below and above) up to z+2R+PD+1 and one slot that is being refilled.  The z window of
// each owned column stays in registers: its lowest planes that are not in the ring are loaded
// from global memory at the start, the rest and every new value come from the ring.  The level t-1 centres of the second-order stencils
// and the coefficients are loaded into registers one plane ahead.  One barrier per plane.
//
// V16 (rows of 16-byte multiples, 16-byte aligned buffers): 16-byte cp.async.cg chunks, the tile
// row widened to whole chunks.  Otherwise: element cp.async.
//
// VX columns per thread, 32 apart (the tile is 32*VX columns wide; a warp's accesses stay on
// consecutive words, free of bank conflicts): VX > 1 shares each thread's per-plane work
// (barrier, staging items, loop control) among VX*2 updates.
// Blocks per SM the register allocation must allow (0: no bound): 2 for the packed FP32 25-point
// factor-grid sweep, whose two column pairs of 2R+1-plane windows take 122 registers.
template <int S, typename T, int VX>
constexpr int naive_min_blocks() { return (S == 4 && sizeof(T) == 4 && VX == 2) ? 2 : 0; }

template <int S, typename T, int TY, int PD, bool V16, int VX>
__global__ void __launch_bounds__(32 * TY, (naive_min_blocks<S, T, VX>())) naive_kernel(const NaiveArgs a) {
  constexpr int R = Traits<S>::R;
  constexpr int NC = Traits<S>::NCOEF;
  constexpr int ROWS = 2 * TY;
  constexpr int A16 = 16 / (int)sizeof(T);
  constexpr int TX = 32 * VX;                  // tile columns
  constexpr int TXW = V16 ? (TX + 2 * R + A16 - 1) / A16 * A16 : TX + 2 * R;  // shared row width
  constexpr int TYW = ROWS + 2 * R, TP = TXW * TYW;
  // ring slots: planes z+R-ZB .. z+2R+PD+1 are live at the update of plane z (R+PD+2+ZB), ZB = 1
  // for the box stencil, whose diagonal neighbours need the x-y tiles of the planes below and above
  constexpr int ZB = Traits<S>::BOX ? 1 : 0;
  constexpr int NP = R + PD + 2 + ZB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);       // [NP][TYW][TXW]
  const T* __restrict__ V = static_cast<const T*>(a.V);
  T* __restrict__ U = static_cast<T*>(a.U);
  const T* __restrict__ coef = static_cast<const T*>(a.coef);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = sizeof(T) == 8 ? static_cast<T>(a.c[i]) : static_cast<T>(a.cf[i]);
  // FP32 with an even number of columns per thread: two columns per packed update (measured at
  // full size: 7-point constant 714 -> 739, red-black 707 -> 738, 25-point factor grid with two
  // columns per thread 284 -> 305 GLUP/s; not the 25-point constant stencil, 328 -> 325; the
  // box stencil packs differently, below).  Radius 4: the thread's columns are adjacent pairs, 64 apart (2 tx,
  // 2 tx + 1, 64 + 2 tx, ...), so that a warp's 8-byte loads of a row stay on consecutive words;
  // otherwise 32 apart.
  constexpr bool PACK = sizeof(T) == 4 && VX % 2 == 0 && !Traits<S>::BOX && S != 2;
  constexpr bool PAIRS = PACK && R == 4;
  constexpr int D2 = PAIRS ? 1 : 32;
  // The box stencil (FP32, two columns per thread) instead gives each thread a 2x2 block of
  // points, rows 2 ty, 2 ty + 1 and columns 2 tx, 2 tx + 1: the block's 4x4x3 neighbourhood is 24
  // aligned 8-byte shared loads (6 per update instead of 24 single loads), and its pairs of
  // columns feed packed updates with one repacked pair per row and plane (320 -> 536 GLUP/s at
  // 512^3).  The same 2x2 block for the 25-point stencils, whose two rows share their y
  // neighbours, was slower (328 -> 304, factor grid 306 -> 279: 118-126 registers, 2 blocks per SM).
  constexpr bool BOX2 = Traits<S>::BOX && sizeof(T) == 4 && VX == 2;
  F2 cst2[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst2[i] = pack2(a.cf[i], a.cf[i]);

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = (int)a.g.nx, ny = (int)a.g.ny, nz = (int)a.g.nz;
  const int ldx = (int)a.g.ldx;
  const int64_t plane = a.g.sy * a.g.ldx;
  const int bx = blockIdx.x * TX, by = blockIdx.y * ROWS;  // padded coords of the tile's corner
  const int z0 = blockIdx.z * a.zc;
  const int nzb = min(a.zc, nz - z0);
  // tile rows/cols that exist in the padded grid
  const int trows = min(TYW, ny + 2 * R - by), tcols = min(TXW, nx + 2 * R - bx);
  const T* Vb = V + (int64_t)z0 * plane + (int64_t)by * ldx + bx;  // padded plane z0, tile corner
  T* Ub = U + (int64_t)(z0 + R) * plane + (int64_t)(by + R) * ldx + (bx + R);

  // This thread's items of one staged plane (fixed for the whole z walk): shared offset within a
  // ring slot and offset within a global plane relative to the tile corner, -1 = none.  An item
  // is one element, or (V16) one 16-byte chunk of a tile row inside the padded row [0, ldx).
  constexpr int W = V16 ? A16 : 1;             // elements per item
  constexpr int NCH = TXW / W;                 // items per tile row
  constexpr int CPT = (NCH * TYW + 32 * TY - 1) / (32 * TY);
  int so[CPT], go[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int i = tid + k * 32 * TY;
    const int r = i / NCH, c = (i - r * NCH) * W;
    const bool ok = i < NCH * TYW && r < trows && (V16 ? bx + c < ldx : c < tcols);
    so[k] = ok ? r * TXW + c : -1;
    go[k] = ok ? r * ldx + c : 0;
  }
  auto copy = [&](T* dst, const T* src) {
    if constexpr (V16) cp_async16_cg(dst, src);
    else cp_async(dst, src);
  };

  // stage padded plane z0 + q (q = 0 .. nzb + 2R - 1) into ring slot q % NP
  auto stage = [&](int q) {
    if (q < nzb + 2 * R) {
      T* dst = ring + (q % NP) * TP;
      const T* src = Vb + (int64_t)q * plane;
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (so[k] >= 0) copy(dst + so[k], src + go[k]);
    }
    cp_async_commit();
  };

  // planes z0+R-ZB .. z0+2R fill the upper windows; planes up to z0 + 2R + PD are staged ahead
  for (int q = R - ZB; q <= 2 * R + PD; ++q) stage(q);

  bool act[2][VX];
  auto row_of = [&](int r) { return BOX2 ? 2 * ty + r : ty + r * TY; };  // the thread's rows
  int cx[VX];  // the thread's columns within the tile
#pragma unroll
  for (int v = 0; v < VX; ++v) cx[v] = PAIRS ? 64 * (v >> 1) + 2 * tx + (v & 1) : (BOX2 ? 2 * tx + v : 32 * v + tx);
  int cofs[2];  // shared offset of column 0 in each of the thread's rows
  T w[2][VX][2 * R + 1];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int row = row_of(r);
    cofs[r] = (row + R) * TXW + R;
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      act[r][v] = (bx + cx[v] < nx) && (by + row < ny);
      // the R-ZB lowest planes of the window, straight from global memory
#pragma unroll
      for (int i = 0; i < R - ZB; ++i)
        w[r][v][i] = act[r][v] ? Vb[(int64_t)i * plane + (row + R) * ldx + R + cx[v]] : T(0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int v = 0; v < VX; ++v)
#pragma unroll
      for (int i = R - ZB; i <= 2 * R; ++i) w[r][v][i] = ring[(i % NP) * TP + cofs[r] + cx[v]];
  // every thread has its first window before the first in-loop staging refills a slot
  __syncthreads();
  // per-column pointers, advanced one plane per update: the output point (also the level t-1
  // centre of the second-order stencils) and coefficient grid 0 of the next plane
  T* up[2][VX];
  const T* kp[2][VX];
  const int64_t gs = a.g.gstride;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const int64_t o = (int64_t)row_of(r) * ldx + cx[v];
      up[r][v] = Ub + o;
      kp[r][v] = coef ? coef + (int64_t)(z0 + R) * plane + (int64_t)(by + R) * ldx + (bx + R) + o : nullptr;
    }
  // coefficients of the first plane, then one plane ahead
  T kv[2][VX][NC > 0 ? NC : 1], kn[2][VX][NC > 0 ? NC : 1];
  if constexpr (NC > 0) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int v = 0; v < VX; ++v) {
#pragma unroll
        for (int g = 0; g < NC; ++g) kn[r][v][g] = act[r][v] ? __ldg(kp[r][v] + g * gs) : T(0);
        kp[r][v] += plane;
      }
  }
  // level t-1 centres (second order): read from the output buffer before this thread overwrites
  // them, one plane ahead (each is read and written by its owning thread only)
  T un[2][VX];
  if constexpr (Traits<S>::ORDER2) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int v = 0; v < VX; ++v) un[r][v] = act[r][v] ? __ldcg(up[r][v]) : T(0);
  }

  for (int zr = 0; zr < nzb; ++zr) {
    const bool more = zr + 1 < nzb;
    if constexpr (NC > 0) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          const bool ld = act[r][v] && more;
#pragma unroll
          for (int g = 0; g < NC; ++g) {
            kv[r][v][g] = kn[r][v][g];
            kn[r][v][g] = ld ? __ldg(kp[r][v] + g * gs) : T(0);
          }
          kp[r][v] += plane;
        }
    }
    T uc[2][VX];
    if constexpr (Traits<S>::ORDER2) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          uc[r][v] = un[r][v];
          un[r][v] = (act[r][v] && more) ? __ldcg(up[r][v] + plane) : T(0);
        }
    }
    const T* tl = ring + ((zr + R) % NP) * TP;  // padded plane z0 + zr + R = interior plane z0 + zr
    const T* tlm = ring + ((zr + R - ZB) % NP) * TP;  // box: the planes below and above
    const T* tlp = ring + ((zr + R + ZB) % NP) * TP;
    if constexpr (BOX2) {
      F2 q[4][3][3];
      const float* pl[3] = {reinterpret_cast<const float*>(tlm), reinterpret_cast<const float*>(tl),
                            reinterpret_cast<const float*>(tlp)};
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
          // shared row 2 ty + rr is tile row 2 ty + rr - 1; shared column 2 tx is column 2 tx - 1
          const float* p = pl[dz] + (2 * ty + rr) * TXW + 2 * tx;
          q[rr][dz][0] = F2{*reinterpret_cast<const unsigned long long*>(p)};
          q[rr][dz][2] = F2{*reinterpret_cast<const unsigned long long*>(p + 2)};
          float a0, a1, b0, b1;
          unpack2(q[rr][dz][0], a0, a1);
          unpack2(q[rr][dz][2], b0, b1);
          q[rr][dz][1] = pack2(a1, b0);
        }
      float res[2][2];
      unpack2(point_update<S, F2>(BoxAcc2<0>{q}, cst2), res[0][0], res[0][1]);
      unpack2(point_update<S, F2>(BoxAcc2<1>{q}, cst2), res[1][0], res[1][1]);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          if (act[r][v]) *up[r][v] = (T)res[r][v];
          up[r][v] += plane;
        }
    } else {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if constexpr (PACK) {
        // columns v and v+1 in one packed update; a column outside the grid is computed from
        // in-bounds shared cells and not stored
#pragma unroll
        for (int v = 0; v < VX; v += 2) {
          if (act[r][v] || act[r][v + 1]) {
            NaiveAcc2<S, TXW, D2> acc{reinterpret_cast<const float*>(tl) + cofs[r] + cx[v],
                                  reinterpret_cast<const float*>(w[r][v]),
                                  reinterpret_cast<const float*>(w[r][v + 1]),
                                  reinterpret_cast<const float*>(kv[r][v]),
                                  reinterpret_cast<const float*>(kv[r][v + 1]),
                                  F2{0},
                                  reinterpret_cast<const float*>(tlm) + cofs[r] + cx[v],
                                  reinterpret_cast<const float*>(tlp) + cofs[r] + cx[v]};
            if constexpr (Traits<S>::ORDER2) acc.uc = pack2((float)uc[r][v], (float)uc[r][v + 1]);
            float res[2];
            unpack2(point_update<S, F2>(acc, cst2), res[0], res[1]);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              if constexpr (Traits<S>::RB)  // red-black: only (x + y + z + t) even is updated
                if ((bx + cx[v + e] + by + ty + r * TY + z0 + zr + a.t) & 1) res[e] = (float)w[r][v + e][R];
              if (act[r][v + e]) *up[r][v + e] = (T)res[e];
            }
          }
        }
#pragma unroll
        for (int v = 0; v < VX; ++v) up[r][v] += plane;
      } else {
#pragma unroll
        for (int v = 0; v < VX; ++v) {
          if (act[r][v]) {
            NaiveAcc<S, T, TXW> acc{tl + cofs[r] + cx[v], w[r][v], kv[r][v], T(0), tlm + cofs[r] + cx[v],
                                    tlp + cofs[r] + cx[v]};
            if constexpr (Traits<S>::ORDER2) acc.uc = uc[r][v];
            T res = point_update<S, T>(acc, cst);
            if constexpr (Traits<S>::RB)  // red-black: only (x + y + z + t) even is updated
              if ((bx + cx[v] + by + ty + r * TY + z0 + zr + a.t) & 1) res = w[r][v][R];
            *up[r][v] = res;
          }
          up[r][v] += plane;
        }
      }
    }
    }
    // advance: stage the plane PD ahead, wait for the next window value, one barrier
    stage(zr + 2 * R + PD + 1);
    cp_async_wait_group<PD>();
    __syncthreads();
    const T* nw = ring + ((zr + 2 * R + 1) % NP) * TP;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int v = 0; v < VX; ++v) {
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) w[r][v][i] = w[r][v][i + 1];
        w[r][v][2 * R] = nw[cofs[r] + cx[v]];
      }
    }
  }
}

// Thread rows per block (each thread owns two rows of the tile): 8, or 4 for the FP64 25-point
// variable stencil, whose 26 coefficient registers per thread allow one 256-thread block per SM
// only; two 128-thread blocks keep the same warps but desynchronise their barriers (measured:
// 16.9 -> 18.4 GLUP/s at 384^3; the other stencils were as fast or faster with 8).
template <int S, typename T>
constexpr int naive_ty() { return (S == 3 && sizeof(T) == 8) ? 4 : 8; }

// Planes staged ahead of use: 4 for the 7-point stencils; for the radius-4 ones, whose planes
// are larger, 2 (25-point constant) or 3 (the stencils with coefficient grids, which also wait
// on their coefficient loads).  Measured at 384^3.
template <int S, typename T>
constexpr int naive_pd() { return Traits<S>::R == 1 ? 4 : (S == 2 ? 2 : 3); }

// Columns per thread (16-byte aligned layouts): 4 for the FP32 7-point constant stencil and 2
// for the FP32 25-point (constant and factor grid) and 27-point box ones, whose sweeps were bound by instruction
// issue (the thread's per-plane work -- barrier, staging items, loop and address bookkeeping --
// is then shared by 2*VX updates: 564 -> 715, 291 -> 336 and 304 -> 320 GLUP/s); else 1 (measured: the FP64
// sweeps are bound by the FP64 pipe, and the stencils with coefficient grids keep a plane of
// coefficients per column in registers, so more columns cost occupancy).
template <int S, typename T, bool V16>
constexpr int naive_vx() {
  return (V16 && sizeof(T) == 4) ? ((S == 0 || S == 6) ? 4 : ((S == 2 || S == 4 || S == 5) ? 2 : 1)) : 1;
}

template <int S, typename T, bool V16>
static size_t naive_smem() {
  constexpr int R = Traits<S>::R, PD = naive_pd<S, T>(), A16 = 16 / (int)sizeof(T);
  constexpr int TX = 32 * naive_vx<S, T, V16>();
  constexpr int TXW = V16 ? (TX + 2 * R + A16 - 1) / A16 * A16 : TX + 2 * R;
  constexpr int NP = R + PD + 2 + (Traits<S>::BOX ? 1 : 0), TP = TXW * (2 * naive_ty<S, T>() + 2 * R);
  return sizeof(T) * (size_t)NP * TP;
}

// Resident blocks per SM of one naive kernel instance (occupancy query, cached per instance).
template <int S, typename T, bool V16>
static int resident_blocks() {
  static int n = -1;
  if (n < 0) {
    const size_t sm = naive_smem<S, T, V16>();
    auto k = naive_kernel<S, T, naive_ty<S, T>(), naive_pd<S, T>(), V16, naive_vx<S, T, V16>()>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 32 * naive_ty<S, T>(), sm) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    n = b;
  }
  return n;
}

template <int S, typename T, bool V16>
static cudaError_t launch_one(const NaiveArgs& a, cudaStream_t st) {
  constexpr int TY = naive_ty<S, T>();
  dim3 block(32, TY);
  constexpr int TX = 32 * naive_vx<S, T, V16>();
  dim3 grid((unsigned)((a.g.nx + TX - 1) / TX), (unsigned)((a.g.ny + 2 * TY - 1) / (2 * TY)),
            (unsigned)((a.g.nz + a.zc - 1) / a.zc));
  const size_t sm = naive_smem<S, T, V16>();
  auto k = naive_kernel<S, T, TY, naive_pd<S, T>(), V16, naive_vx<S, T, V16>()>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, sm, st>>>(a);
  return cudaGetLastError();
}

template <int S, typename T>
static cudaError_t launch_v(const NaiveArgs& a, cudaStream_t st) {
  return a.v16 ? launch_one<S, T, true>(a, st) : launch_one<S, T, false>(a, st);
}

int naive_tile_y(int stencil, int dtype) {
  const bool f64 = dtype == GIRIH_F64;
  auto pick = [&](auto s_tag) -> int {
    constexpr int S = decltype(s_tag)::value;
    return 2 * (f64 ? naive_ty<S, double>() : naive_ty<S, float>());
  };
  switch (stencil) {
    case 0: return pick(std::integral_constant<int, 0>());
    case 1: return pick(std::integral_constant<int, 1>());
    case 2: return pick(std::integral_constant<int, 2>());
    case 3: return pick(std::integral_constant<int, 3>());
    case 4: return pick(std::integral_constant<int, 4>());
    case 5: return pick(std::integral_constant<int, 5>());
    default: return pick(std::integral_constant<int, 6>());
  }
}

int naive_tile_x(int stencil, int dtype, bool v16) {
  const bool f64 = dtype == GIRIH_F64;
  auto pick = [&](auto s_tag) -> int {
    constexpr int S = decltype(s_tag)::value;
    if (f64) return 32 * (v16 ? naive_vx<S, double, true>() : naive_vx<S, double, false>());
    return 32 * (v16 ? naive_vx<S, float, true>() : naive_vx<S, float, false>());
  };
  switch (stencil) {
    case 0: return pick(std::integral_constant<int, 0>());
    case 1: return pick(std::integral_constant<int, 1>());
    case 2: return pick(std::integral_constant<int, 2>());
    case 3: return pick(std::integral_constant<int, 3>());
    case 4: return pick(std::integral_constant<int, 4>());
    case 5: return pick(std::integral_constant<int, 5>());
    default: return pick(std::integral_constant<int, 6>());
  }
}

int naive_resident_blocks(int stencil, int dtype, bool v16) {
  const bool f64 = dtype == GIRIH_F64;
  auto pick = [&](auto s_tag) -> int {
    constexpr int S = decltype(s_tag)::value;
    if (f64) return v16 ? resident_blocks<S, double, true>() : resident_blocks<S, double, false>();
    return v16 ? resident_blocks<S, float, true>() : resident_blocks<S, float, false>();
  };
  switch (stencil) {
    case 0: return pick(std::integral_constant<int, 0>());
    case 1: return pick(std::integral_constant<int, 1>());
    case 2: return pick(std::integral_constant<int, 2>());
    case 3: return pick(std::integral_constant<int, 3>());
    case 4: return pick(std::integral_constant<int, 4>());
    case 5: return pick(std::integral_constant<int, 5>());
    default: return pick(std::integral_constant<int, 6>());
  }
}

// z planes per block, 16 to 64: the chunk count that maximises (fraction of the last wave of
// blocks that is used) x (fraction of each block's staged planes that it updates, zc/(zc+2R)),
// i.e. fills the device's resident block slots in whole waves without re-reading too many
// z-halo planes (fewer chunks on ties).
int naive_z_chunk(int64_t nx, int64_t ny, int64_t nz, int R, int tile_x, int tile_y, int resident_per_sm,
                  int sm_count) {
  const int64_t tiles = ((nx + tile_x - 1) / tile_x) * ((ny + tile_y - 1) / tile_y);
  const int64_t slots = (int64_t)std::max(resident_per_sm, 1) * std::max(sm_count, 1);
  const int64_t cmin = std::max<int64_t>((nz + 63) / 64, 1), cmax = std::max<int64_t>((nz + 15) / 16, cmin);
  int64_t best_c = cmin;
  double best_eff = -1.0;
  for (int64_t c = cmin; c <= cmax; ++c) {
    const int64_t zc = (nz + c - 1) / c;
    const int64_t blocks = tiles * ((nz + zc - 1) / zc);
    const double waves = (double)blocks / (double)slots;
    const double eff = waves / std::ceil(waves) * (double)zc / (double)(zc + 2 * R);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best_c = c;
    }
  }
  return (int)((nz + best_c - 1) / best_c);
}

cudaError_t launch_naive_step(int stencil, int dtype, const NaiveArgs& a, cudaStream_t st) {
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case 0: return f64 ? launch_v<0, double>(a, st) : launch_v<0, float>(a, st);
    case 1: return f64 ? launch_v<1, double>(a, st) : launch_v<1, float>(a, st);
    case 2: return f64 ? launch_v<2, double>(a, st) : launch_v<2, float>(a, st);
    case 3: return f64 ? launch_v<3, double>(a, st) : launch_v<3, float>(a, st);
    case 4: return f64 ? launch_v<4, double>(a, st) : launch_v<4, float>(a, st);
    case 5: return f64 ? launch_v<5, double>(a, st) : launch_v<5, float>(a, st);
    default: return f64 ? launch_v<6, double>(a, st) : launch_v<6, float>(a, st);
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
