// Wavefront-diamond sweep with neighbour-only synchronisation (variant RELAXED_PERSISTENT): the
// tiling, wavefront and persistent FIFO schedule of the FED_PERSISTENT kernel (mwd_vec.cuh,
// Sects. 4.2.1 and 4.2.3), with the per-step synchronisation reduced to what the data flow needs
// and the data movement taken off the computing warps.
//
// Synchronisation.  A wavefront step of a tile needs, besides the block's own results of the
// previous step, only the x-halo columns its two neighbours in the cluster computed in that step.
// Those arrive as asynchronous remote stores (st.async) that count their bytes on a halo mbarrier
// of the receiving block, which waits for exactly that many bytes: the relaxed synchronisation
// of Sect. 4.2.1 (a thread group member waits for its neighbour, not for the whole group), here
// along x where the halo exchange goes both ways.  No cluster-wide barrier and no release fence
// is taken per step (a cluster barrier is taken once per tile).  One plane per level and step
// (nf = 1): then a block can run at most one step ahead of a neighbour, and a push of step w+1
// (planes w+1 - s*K of level s) never meets a value the receiver still reads in step w (level
// s-1 reads its x neighbours at planes w - (s-1)*K = w + 1 - s*K + 1).
//
// Warp roles.  The computing warps own tasks (level s, row pair y0/y0+1, one 16-byte vector of
// columns) for the whole tile; a task keeps planes z-1 and z of its two rows in registers and per
// plane reads plane z+1 of its rows, rows y0-1 and y0+2 of plane z and the two x neighbours of
// each row from shared memory, and writes two 16-byte vectors.  A value that no later level of
// the tile overwrites (level t + 2 does not cover the row) is final: the task also stores it to
// global memory, so there is no separate write-back pass and the halo is never written.  The last
// warp stages planes with the bulk-copy (TMA) engine: one tensor copy per buffer and plane (a box
// of YW rows x XT columns, the slab and its halo), completing on one of eight load mbarriers
// (global step modulo 8), LEAD steps ahead of use.  Step w (named barriers FULL and DONE):
//   computing warps:  wait FULL(w); update and store; proxy fence (results -> later bulk copies
//     into the same slots); arrive DONE(w)
//   mover, iteration w (overlapping the computing warps' step w):  wait DONE(w-1); stage the
//     plane first read at step w+L; wait for the staging of step w+2 and for the neighbours'
//     halo bytes of step w; arrive FULL(w+1).
// Staging two steps ahead of need means a plane has landed before any neighbour (at most one
// step ahead) can push into it.
//
// Ring depth: a slot is restaged once its previous plane is below every level's read window in
// the step being computed:  NZ = L + 2R + 1 + smax K,  K = R + 1, smax = H - 2,  L = lead (3..8).
// Planes are padded to 128 bytes (the tensor copies' destination alignment).
//
// Radius-1 first-order stencils (7-point constant, 7-point variable, red-black Gauss-Seidel) on
// rows of 16-byte multiples with 16-byte aligned buffers.  Every point goes through point_update
// (stencil.cuh), so the result equals the naive sweep bit for bit.
#pragma once
#include <type_traits>

#include "mwd_kernel.cuh"

namespace girih {

// Accessor of one point of a task: row ROW (0: y0, 1: y0+1) and column I of the vector (both
// compile-time after unrolling, so every access is a register):
//   yr[0..3]  rows y0-1 .. y0+2 of plane z;  zm[ROW], zp[ROW]  planes z-1, z+1 of the row;
//   xm[ROW], xp[ROW]  the columns left and right of the vector;  kv[g]  coefficient grid g of the row.
template <typename T, int VX, int ROW, int I>
struct TaskAcc {
  const T (*yr)[VX];
  const T (*zm)[VX];
  const T (*zp)[VX];
  const T* xm;
  const T* xp;
  const T (*kv)[VX];
  __device__ __forceinline__ T c() const { return yr[1 + ROW][I]; }
  __device__ __forceinline__ T x(int d) const {
    return d < 0 ? (I == 0 ? xm[ROW] : yr[1 + ROW][I - 1]) : (I == VX - 1 ? xp[ROW] : yr[1 + ROW][I + 1]);
  }
  __device__ __forceinline__ T y(int d) const { return yr[1 + ROW + d][I]; }
  __device__ __forceinline__ T z(int d) const { return d < 0 ? zm[ROW][I] : zp[ROW][I]; }
  __device__ __forceinline__ T u() const { return T(0); }
  __device__ __forceinline__ T k(int g) const { return kv[g][I]; }
};

// The VX points of row ROW of a task.
template <int S, typename T, int VX, int ROW, int I>
__device__ __forceinline__ void task_row(const T (*yr)[VX], const T (*zm)[VX], const T (*zp)[VX], const T* xm,
                                         const T* xp, const T (*kv)[VX], const T* cst, T* r) {
  if constexpr (I < VX) {
    const TaskAcc<T, VX, ROW, I> acc{yr, zm, zp, xm, xp, kv};
    r[I] = point_update<S, T>(acc, cst);
    task_row<S, T, VX, ROW, I + 1>(yr, zm, zp, xm, xp, kv, cst, r);
  }
}

// As TaskAcc, with the coefficients of both rows: kv[g][ROW][i].
template <typename T, int VX, int ROW, int I>
struct TaskAcc2 {
  const T (*yr)[VX];
  const T (*zm)[VX];
  const T (*zp)[VX];
  const T* xm;
  const T* xp;
  const T (*kv)[2][VX];
  __device__ __forceinline__ T c() const { return yr[1 + ROW][I]; }
  __device__ __forceinline__ T x(int d) const {
    return d < 0 ? (I == 0 ? xm[ROW] : yr[1 + ROW][I - 1]) : (I == VX - 1 ? xp[ROW] : yr[1 + ROW][I + 1]);
  }
  __device__ __forceinline__ T y(int d) const { return yr[1 + ROW + d][I]; }
  __device__ __forceinline__ T z(int d) const { return d < 0 ? zm[ROW][I] : zp[ROW][I]; }
  __device__ __forceinline__ T u() const { return T(0); }
  __device__ __forceinline__ T k(int g) const { return kv[g][ROW][I]; }
};
template <int S, typename T, int VX, int ROW, int I>
__device__ __forceinline__ void task_row2(const T (*yr)[VX], const T (*zm)[VX], const T (*zp)[VX], const T* xm,
                                          const T* xp, const T (*kv)[2][VX], const T* cst, T* r) {
  if constexpr (I < VX) {
    const TaskAcc2<T, VX, ROW, I> acc{yr, zm, zp, xm, xp, kv};
    r[I] = point_update<S, T>(acc, cst);
    task_row2<S, T, VX, ROW, I + 1>(yr, zm, zp, xm, xp, kv, cst, r);
  }
}

// Coefficient grids 0 .. NC-1 of one row's VX columns: 16-byte read-only loads.
template <typename T, int VX, int NC>
__device__ __forceinline__ void load_coef(const T* kp, int64_t gstride, T (*kv)[VX]) {
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const V16 k = __ldg(reinterpret_cast<const V16*>(kp + q * gstride));
    if constexpr (sizeof(T) == 4) {
      kv[q][0] = k.x; kv[q][1] = k.y; kv[q][2] = k.z; kv[q][3] = k.w;
    } else {
      kv[q][0] = k.x; kv[q][1] = k.y;
    }
  }
}

// Coefficient grids 0 .. NC-1 of two rows (row y0 at kp, row y0+1 at kp + ldx): kv[g][row][i].
template <typename T, int VX, int NC>
__device__ __forceinline__ void load_coef_pair(const T* kp, int64_t gstride, int ldx, T (*kv)[2][VX]) {
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const V16 k = __ldg(reinterpret_cast<const V16*>(kp + q * gstride + r * ldx));
      if constexpr (sizeof(T) == 4) {
        kv[q][r][0] = k.x; kv[q][r][1] = k.y; kv[q][r][2] = k.z; kv[q][r][3] = k.w;
      } else {
        kv[q][r][0] = k.x; kv[q][r][1] = k.y;
      }
    }
}

__device__ __forceinline__ void st_async_push(uint32_t addr, float v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v),
               "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void st_async_push(uint32_t addr, double v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v),
               "r"(mbar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, "
      "p; }"
      : "=r"(ok)
      : "r"(m), "r"(parity)
      : "memory");
  return ok != 0;
}

// Named barrier ID (1..15; 0 is __syncthreads) over n threads: wait for all, or arrive only.  The
// id is an immediate, so the kernel reserves only the barriers it uses.
template <int ID>
__device__ __forceinline__ void nbar_sync(int n) { asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(n) : "memory"); }
template <int ID>
__device__ __forceinline__ void nbar_arrive(int n) { asm volatile("bar.arrive %0, %1;" ::"n"(ID), "r"(n) : "memory"); }
// The block's barriers between its computing warps and its mover warp: FULL(w) (inputs of step w
// ready, ids 1-2 by step parity) and DONE(w) (step w computed, ids 3-4).  Alternating ids keep a
// producer's arrival for step w+1 from counting towards step w.
__device__ __forceinline__ void sync_full(int w, int n) {
  if (w & 1) nbar_sync<2>(n);
  else nbar_sync<1>(n);
}
__device__ __forceinline__ void arrive_full(int w, int n) {
  if (w & 1) nbar_arrive<2>(n);
  else nbar_arrive<1>(n);
}
__device__ __forceinline__ void sync_done(int w, int n) {
  if (w & 1) nbar_sync<4>(n);
  else nbar_sync<3>(n);
}
__device__ __forceinline__ void arrive_done(int w, int n) {
  if (w & 1) nbar_arrive<4>(n);
  else nbar_arrive<3>(n);
}
constexpr int kMovers = 32;  // the block's last warp moves data; the others compute
constexpr int kLoadBars = 8;  // mbarriers of the staging copies, by global step modulo 8 (lead <= 8)


__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Halo pushes a block receives per step: from its left neighbour if that one's slab is full (it
// then pushes its last column), from its right neighbour if it has columns (its first column).
__device__ __forceinline__ int halo_senders(int nx, int XW, int C, int rank) {
  const int x0 = rank * XW - 1;
  return ((C > 1 && rank > 0 && nx - (x0 - XW) >= XW) ? 1 : 0) + ((C > 1 && rank < C - 1 && nx - (x0 + XW) > 0) ? 1 : 0);
}

// Tensor copy of box (x, y, z) of a 3D tensor map into shared memory, completing on mbar.  x may
// be negative or past the end (filled with zeros); x * element size is a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(mbar))
      : "memory");
}

// Bounded wait of all lanes of a warp on an mbarrier phase; a timeout sets the error word.
__device__ __forceinline__ void warp_wait_phase(uint32_t mb, uint32_t parity, int* err) {
  if (!mbar_try_wait_cluster(mb, parity)) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_cluster(mb, parity)) {
      if (global_ns() - t0 > kMbarWaitNs) {
        atomicOr(err, GIRIH_ETIMEOUT);
        break;
      }
    }
  }
  __syncwarp();
}

// One tile (diamond (a, a - rho), this block's x slab) from staging to write-back.  gstep: wavefront
// steps the block has run in earlier tiles of this launch; the halo and load mbarriers serve
// global steps in turn (halo: by parity, loads: modulo kLoadBars), one phase per step.
template <int S, typename T, int G>
__device__ __forceinline__ void mwd_async_tile(const MwdArgs& A, const int rho, const int a, int& gstep) {
  static_assert(Traits<S>::R == 1 && !Traits<S>::ORDER2 && !Traits<S>::BOX, "radius-1 first-order stencils");
  constexpr int R = 1;
  constexpr int NC = Traits<S>::NCOEF;
  constexpr int NCO = NC > 0 ? NC : 1;
  constexpr int A16 = 16 / (int)sizeof(T);
  constexpr int VX = A16;  // one 16-byte vector per task
  constexpr int HM = A16;  // shared column of the slab's first column (R rounded up to 16 bytes)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, K = A.K;
  const int L = A.lead;  // steps between a plane's staging and its first use
  const int pe = A.PE;  // elements per plane slot: YW * XT rounded up to 128 bytes
  const int be = NZ * pe;
  const int ring = be;
  uint64_t* hb = reinterpret_cast<uint64_t*>(smem_raw + (((size_t)2 * be * sizeof(T) + 15) / 16) * 16);
  uint64_t* lb = hb + 2;
  int* lev_lo = reinterpret_cast<int*>(lb + kLoadBars);
  int* lev_w = lev_lo + A.H;
  int* lev_pp = lev_w + A.H;

  const int nx = (int)A.g.nx, ny = (int)A.g.ny, nz = (int)A.g.nz;
  const int ldx = (int)A.g.ldx;
  const int64_t gplane = A.g.sy * A.g.ldx;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const int dw = A.dw;
  const int b = a - rho;
  const int P0 = a * dw - rho * (dw / 2);
  const int Y0 = P0 - R;
  const int pc0 = rank * XW;  // padded column of slab column 0
  const int x0 = pc0 - R;     // its interior column
  const int vlo = max(0, -x0);
  const int vhi = min(XW, nx - x0);
  const bool active = vhi > vlo;
  const int Hh = A.H / 2;
  const int tb = max((rho - 1) * Hh + 1, 0);
  const int te = min((rho + 1) * Hh - 1, A.T - 1);
  if (tb > te) return;  // uniform over the cluster
  const int nlev = te - tb + 1, smax = nlev - 1;
  const int NT = blockDim.x, tid = threadIdx.x;
  const int NTc = NT - kMovers;
  const bool mover = tid >= NTc;
  const int lane = tid & 31;
  const int npush_in = halo_senders(nx, XW, C, rank);
  const uint32_t hb0 = smem_addr(&hb[0]);
  const uint32_t lb0 = smem_addr(&lb[0]);
  const int g0 = gstep;         // global step of this tile's step 0
  const int W = nz + smax * K;  // wavefront steps (one plane per level and step)
  gstep += W;

  if (tid == 0) {
    int acc = 0;
    for (int s = 0; s < nlev; ++s) {
      const int t = tb + s;
      const int lo = max(lev_lo_of(a, b, dw, R, t), 0);
      const int hi = min(lev_hi_of(a, b, dw, R, t), ny);
      lev_lo[s] = lo;
      lev_w[s] = max(hi - lo, 0);
      lev_pp[s] = acc;
      acc += (max(hi - lo, 0) + 1) / 2;
    }
    lev_pp[nlev] = acc;
  }
  __syncthreads();
  // halo bytes one neighbour pushes in step w: one element per row of every level whose plane of
  // step w lies in [0, nz)
  auto halo_bytes = [&](int w) -> uint32_t {
    uint32_t n = 0;
    for (int s = 0; s < nlev; ++s) {
      const int z = w - s * K;
      if (z >= 0 && z < nz) n += (uint32_t)lev_w[s];
    }
    return n * (uint32_t)npush_in * (uint32_t)sizeof(T);
  };

  // ---- mover: the staging copies of tile step j (planes -R .. R for step 0, plane j + R for step
  //      j >= 1: the planes level 0 newly reads), both buffers, completing on load mbarrier
  //      (g0 + j) mod kLoadBars ----
  const uint32_t box_bytes = (uint32_t)(YW * XT * (int)sizeof(T));
  auto stage_step = [&](int j) {
    const int zlo = j == 0 ? -R : j + R, zhi = j + R;
    int np = 0;
    for (int z = zlo; z <= zhi; ++z) np += (z >= -R && z < nz + R && active) ? 1 : 0;
    uint64_t* m = &lb[(g0 + j) % kLoadBars];
    if (lane == 0) {
      mbar_expect_tx(m, (uint32_t)np * 2u * box_bytes);
      for (int z = zlo; z <= zhi; ++z) {
        if (z < -R || z >= nz + R || !active) continue;
        const int slot = (z + R) % NZ;
        tma_load_3d(sm + slot * pe, &A.tm[0], pc0 - HM, Y0 + R, z + R, m);
        tma_load_3d(sm + be + slot * pe, &A.tm[1], pc0 - HM, Y0 + R, z + R, m);
      }
    }
    __syncwarp();
  };
  auto wait_step = [&](int j) {  // all lanes: the staging of tile step j has landed
    const int gs = g0 + j;
    warp_wait_phase(lb0 + (uint32_t)((gs % kLoadBars) * 8), (uint32_t)((gs / kLoadBars) & 1), A.err);
  };

  // ---- computing threads: tasks (level s, row pair, 16-byte vector), owned for the tile, each
  //      with a register window of planes z-1 and z of its two rows ----
  int t_in[G], t_out[G], t_z[G], t_po[G], t_fl[G], t_par[G];
  const T* t_k[G];
  T* t_g[G];
  T t_zm[G][2][VX], t_zc[G][2][VX];
  // coefficient grids of the task's plane, loaded one step ahead (variable-coefficient stencils):
  // the read-only loads of plane z+1 are in flight while the block synchronises and computes
  T t_kn[G][NC > 0 ? NC : 1][NC > 0 ? 2 : 1][VX];
  if (!mover) {
    const int npairs = lev_pp[nlev];
    const int nvec = XW / VX;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int id = tid + g * NTc;
      const int pr = id / nvec, xl = (id - pr * nvec) * VX;
      const bool valid = active && pr < npairs && xl + VX > vlo && xl < vhi;
      int s = 0;
      if (valid)
        while (lev_pp[s + 1] <= pr) ++s;
      const int y0 = valid ? lev_lo[s] + 2 * (pr - lev_pp[s]) : 0;
      const int t = tb + s;
      const int ro = (y0 - Y0) * XT + HM + xl;
      t_in[g] = (t & 1) * be + ro;
      t_out[g] = ((t & 1) ^ 1) * be + ro;
      t_z[g] = -s * K;
      t_po[g] = (((-s * K + R) % NZ + NZ) % NZ) * pe;
      const int lo = max(0, vlo - xl), hi = min(VX, vhi - xl);
      const bool row1 = valid && (y0 + 1 < lev_lo[s] + lev_w[s]);
      // a row's value of level t+1 is final in the tile unless level t+2 also updates the row
      auto covers = [&](int y, int tt) {
        return tt <= te && y >= max(lev_lo_of(a, b, dw, R, tt), 0) && y < min(lev_hi_of(a, b, dw, R, tt), ny);
      };
      const bool fin0 = valid && !covers(y0, t + 2), fin1 = row1 && !covers(y0 + 1, t + 2);
      // bits: 0 valid, 1 second row, 2 push left, 3 push right, 4 partial vector, 5 window
      // loaded, 6 row y0 final, 7 row y0+1 final, 8.. lo, 12.. hi
      t_fl[g] = (valid ? 1 : 0) | (row1 ? 2 : 0) | ((valid && C > 1 && rank > 0 && xl < R) ? 4 : 0) |
                ((valid && C > 1 && rank < C - 1 && vhi == XW && xl + VX > XW - R) ? 8 : 0) |
                ((lo != 0 || hi != VX) ? 16 : 0) | (fin0 ? 64 : 0) | (fin1 ? 128 : 0) | (lo << 8) | (hi << 12);
      t_g[g] = static_cast<T*>(((t + 1) & 1) ? A.buf1 : A.buf0) + (int64_t)(-s * K + R) * gplane +
               (int64_t)(y0 + R) * ldx + (pc0 + xl);
      t_par[g] = (x0 + xl + y0 + t) & 1;
      t_k[g] = NC ? static_cast<const T*>(A.coef) + (int64_t)(-s * K + R) * gplane + (int64_t)(y0 + R) * ldx +
                        (pc0 + xl)
                  : nullptr;
    }
  }
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = sizeof(T) == 8 ? static_cast<T>(A.c[i]) : static_cast<T>(A.cf[i]);
  const int64_t gstride = A.g.gstride;
  const uint32_t sm_u32 = smem_addr(sm);
  const uint32_t left_base = (C > 1 && rank > 0) ? map_to_rank(sm_u32, rank - 1) : 0u;
  const uint32_t right_base = (C > 1 && rank < C - 1) ? map_to_rank(sm_u32, rank + 1) : 0u;
  const uint32_t left_hb = (C > 1 && rank > 0) ? map_to_rank(hb0, rank - 1) : 0u;
  const uint32_t right_hb = (C > 1 && rank < C - 1) ? map_to_rank(hb0, rank + 1) : 0u;

  // ---- prologue (mover): arm the halo phases of steps 0 and 1 (the previous tile waited for
  //      every phase it used), request the planes of steps 0 .. L-1, wait for steps 0 and 1 ----
  if (mover) {
    if (lane == 0 && npush_in) {
      mbar_expect_tx(&hb[g0 & 1], halo_bytes(0));
      if (W > 1) mbar_expect_tx(&hb[(g0 + 1) & 1], halo_bytes(1));
    }
    fence_proxy_async_global();  // global data acquired before this tile -> bulk loads
    for (int j = 0; j < L && j < W; ++j) stage_step(j);
    wait_step(0);
    if (W > 1) wait_step(1);
  }
  // all blocks' halo mbarriers are armed, and the first planes visible
  __syncwarp();
  cluster_barrier();

  if (!mover) {
    for (int w = 0; w < W; ++w) {
      __syncwarp();  // the named barriers are warp-aligned instructions
      if (w > 0) sync_full(w, NT);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int fl = t_fl[g];
        const int z = t_z[g] + w;
        const int po = t_po[g];
        t_po[g] = (po + pe == ring) ? 0 : po + pe;  // the task's plane of step w+1
        const T* kp = t_k[g];
        if constexpr (NC > 0) t_k[g] += gplane;
        T* gp = t_g[g];
        t_g[g] += gplane;
        if (!(fl & 1) || z < 0 || z >= nz) continue;
        const T* Vb = sm + t_in[g];
        const T* P = Vb + po;
        const bool row1 = fl & 2;
        if (!(fl & 32)) {  // first plane of the task: load the window (planes z-1, z)
          const int pm = (po == 0 ? ring : po) - pe;
          lds_vec<T, VX>(Vb + pm, t_zm[g][0]);
          lds_vec<T, VX>(Vb + pm + XT, t_zm[g][1]);
          lds_vec<T, VX>(P, t_zc[g][0]);
          lds_vec<T, VX>(P + XT, t_zc[g][1]);
          t_fl[g] |= 32;
        }
        const int pp = (po + pe == ring) ? 0 : po + pe;
        T yr[4][VX], zp[2][VX], xm[2], xp[2];
        lds_vec<T, VX>(P - XT, yr[0]);
        // without a second row, row y0+2 may lie past the tile: read row y0+1 instead
        lds_vec<T, VX>(P + (row1 ? 2 * XT : XT), yr[3]);
        lds_vec<T, VX>(Vb + pp, zp[0]);
        lds_vec<T, VX>(Vb + pp + XT, zp[1]);
        xm[0] = P[-1];
        xp[0] = P[VX];
        xm[1] = P[XT - 1];
        xp[1] = P[XT + VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) {
          yr[1][i] = t_zc[g][0][i];
          yr[2][i] = t_zc[g][1][i];
        }
        T r0[VX], r1[VX];
        if constexpr (NC > 0) {
          if (!(fl & 32)) load_coef_pair<T, VX, NC>(kp, gstride, ldx, t_kn[g]);  // first plane: not prefetched
          task_row2<S, T, VX, 0, 0>(yr, t_zm[g], zp, xm, xp, t_kn[g], cst, r0);
          task_row2<S, T, VX, 1, 0>(yr, t_zm[g], zp, xm, xp, t_kn[g], cst, r1);
          // prefetch the next plane's coefficients: consumed in the next step, so the loads are in
          // flight while the block finishes this step and synchronises
          if (z + 1 < nz) load_coef_pair<T, VX, NC>(kp + gplane, gstride, ldx, t_kn[g]);
        } else {
          T kv[1][VX];
          task_row<S, T, VX, 0, 0>(yr, t_zm[g], zp, xm, xp, kv, cst, r0);
          task_row<S, T, VX, 1, 0>(yr, t_zm[g], zp, xm, xp, kv, cst, r1);
        }
        if constexpr (Traits<S>::RB) {
          // red-black: only points with (x + y + z + t) even are updated (row y0+1 has the other
          // colour); the others keep their value
#pragma unroll
          for (int i = 0; i < VX; ++i) {
            const bool odd0 = (t_par[g] + i + z) & 1;
            if (odd0) r0[i] = yr[1][i];
            else r1[i] = yr[2][i];
          }
        }
        T* Ub = sm + t_out[g] + po;
        if (!(fl & 16)) {
          sts_vec<T, VX>(Ub, r0);
          if (row1) sts_vec<T, VX>(Ub + XT, r1);
          if (fl & 64) sts_vec<T, VX>(gp, r0);  // final values go to global memory as well
          if (fl & 128) sts_vec<T, VX>(gp + ldx, r1);
        } else {
          const int lo = (fl >> 8) & 15, hi = (fl >> 12) & 15;
#pragma unroll
          for (int i = 0; i < VX; ++i)
            if (i >= lo && i < hi) {
              Ub[i] = r0[i];
              if (row1) Ub[XT + i] = r1[i];
              if (fl & 64) gp[i] = r0[i];
              if (fl & 128) gp[ldx + i] = r1[i];
            }
        }
        if (fl & 12) {  // x-halo pushes of this step (counted on the neighbour's halo mbarrier)
          const uint32_t so = (uint32_t)(t_out[g] + po) * (uint32_t)sizeof(T);
          if (fl & 4) {  // first column -> left neighbour's right halo column
            const uint32_t oi = so + (uint32_t)(XW * (int)sizeof(T));
            const uint32_t mb = left_hb + (uint32_t)(((g0 + w) & 1) * 8);
            st_async_push(left_base + oi, r0[0], mb);
            if (row1) st_async_push(left_base + oi + (uint32_t)(XT * (int)sizeof(T)), r1[0], mb);
          }
          if (fl & 8) {  // last column -> right neighbour's left halo column
            const uint32_t oi = so + (uint32_t)((VX - 1) * (int)sizeof(T)) - (uint32_t)(XW * (int)sizeof(T));
            const uint32_t mb = right_hb + (uint32_t)(((g0 + w) & 1) * 8);
            st_async_push(right_base + oi, r0[VX - 1], mb);
            if (row1) st_async_push(right_base + oi + (uint32_t)(XT * (int)sizeof(T)), r1[VX - 1], mb);
          }
        }
        // slide the window one plane up
#pragma unroll
        for (int i = 0; i < VX; ++i) {
          t_zm[g][0][i] = t_zc[g][0][i];
          t_zm[g][1][i] = t_zc[g][1][i];
          t_zc[g][0][i] = zp[0][i];
          t_zc[g][1][i] = zp[1][i];
        }
      }
      fence_proxy_async_shared();  // shared-memory results ordered before later bulk copies into the slots
      __syncwarp();
      arrive_done(w, NT);
    }
  } else {
    for (int it = 0; it < W; ++it) {
      if (it > 0) {
        __syncwarp();
        sync_done(it - 1, NT);
      }
      if (it + L < W) stage_step(it + L);
      if (it + 2 < W) wait_step(it + 2);
      if (npush_in) {
        const int gs = g0 + it;
        warp_wait_phase(hb0 + (uint32_t)((gs & 1) * 8), (uint32_t)((gs >> 1) & 1), A.err);
        // every lane has seen the phase of step it complete: arm the mbarrier for step it+2
        if (lane == 0 && it + 2 < W) mbar_expect_tx(&hb[gs & 1], halo_bytes(it + 2));
      }
      __syncwarp();
      if (it + 1 < W) arrive_full(it + 1, NT);
    }
    __syncwarp();
    if (W > 0) sync_done(W - 1, NT);
  }
}

// Persistent kernel: every cluster of a grid that fits the device at once takes diamonds from the
// FIFO in row-major order and starts one once its two parents in the previous row have published
// completion (the runtime of Sect. 4.2.3; same protocol as mwd_vec_kernel's persistent mode).  The
// cluster barrier after a tile orders every block's stores of final values (release) before rank
// 0 publishes the flag.
template <int S, typename T, int G>
__global__ void __launch_bounds__(async_max_threads(G, Traits<S>::NCOEF > 0), 1)
    mwd_async_kernel(const __grid_constant__ MwdArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C = A.C;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const size_t ring_bytes = (((size_t)2 * A.NZ * A.PE * sizeof(T) + 15) / 16) * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes);
  int* slot = reinterpret_cast<int*>(bars + 2 + kLoadBars) + 3 * A.H + 1;
  // the halo and load mbarriers, initialised once per launch (the first cluster barrier below
  // orders the initialisation before any neighbour's push or bulk copy)
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 + kLoadBars; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x == blockDim.x - 1) {  // the mover's tensor-map descriptors, fetched once
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tm[0])) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tm[1])) : "memory");
  }
  int gstep = 0;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const int it = atomicAdd(A.fifo, 1);
      for (int r = 0; r < C; ++r) st_cluster_u32(map_to_rank(smem_addr(slot), (uint32_t)r), (uint32_t)it);
    }
    __syncwarp();
    cluster_barrier();
    const int it = *reinterpret_cast<volatile int*>(slot);
    if (it >= A.n_items) break;
    const int rho = A.items[2 * it], a = A.items[2 * it + 1];
    if (rank == 0 && threadIdx.x == 0 && rho > 0) {
      const int first = A.rows[3 * (rho - 1)], amin = A.rows[3 * (rho - 1) + 1], nd = A.rows[3 * (rho - 1) + 2];
      const uint64_t t0 = global_ns();
      const bool gave_up = *reinterpret_cast<volatile int*>(A.err) != 0;
      for (int d = a - 1; d <= a && !gave_up; ++d) {
        if (d < amin || d >= amin + nd) continue;
        const int* f = A.flags + first + (d - amin);
        int v;
        for (;;) {
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
          if (v == A.epoch) break;
          if (global_ns() - t0 > kMbarWaitNs) {
            atomicOr(A.err, GIRIH_ETIMEOUT);
            break;
          }
        }
      }
    }
    __syncwarp();
    cluster_barrier();
    mwd_async_tile<S, T, G>(A, rho, a, gstep);
    __syncwarp();
    cluster_barrier();
    if (rank == 0 && threadIdx.x == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(A.flags + it), "r"(A.epoch) : "memory");
    }
  }
}

}  // namespace girih
