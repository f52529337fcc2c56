// Multi-threaded wavefront-diamond sweep (MWD, arXiv 1510.04995, Sect. 4.2.1), GB300 form.
//
// Tiling (Sects. 2.1.2, 3.2).  Updates are points (y, t) of the y-t plane (update t makes level
// t+1).  Diamond (a, b) holds the updates with  a*Dw <= y + R*t < (a+1)*Dw  and
// b*Dw <= y - R*t < (b+1)*Dw: a tiling by the two families of lines of slope +-R.  An update
// depends only on updates of the same diamond or of diamonds (a-1, b), (a, b+1), (a-1, b+1);
// so the diamonds of one row rho = a - b are independent and rows run in order, one launch per
// row.  Row rho spans the steps t with (rho-1)*Dw < 2*R*t < (rho+1)*Dw (H-1 levels, H = Dw/R)
// and its diamonds' y projections [(a+b)*Dw/2, (a+b+2)*Dw/2) partition y.
//
// Two buffers, updated in place (Listing 3's pointer swap generalised): level t of a point lives
// in buffer t%2.  Writing level t+1 overwrites level t-1, whose readers are exactly the updates
// level t+1 depends on, so any dependency-respecting order is race free; this holds for the
// global arrays and for the shared-memory copy of a tile alike.
//
// Tile = extruded diamond (full z) x x-slab, one thread block per slab, the slabs of one diamond
// forming a thread-block cluster (the paper's thread group, Sect. 4.1, sharing one tile; the
// x split is the balanced x decomposition of Listing 5).  Each block keeps a ring of z planes of
// both buffers in shared memory: [2][NZ][YW = Dw + 2R][XT >= XW + 2R].  The wavefront walks up in
// z (Sect. 2.1.1): at step w, local level s updates planes [w*nf - s*K, w*nf - s*K + nf) with the
// level skew K = R + nf, which makes every input of a step come from earlier steps, so one
// synchronisation per step suffices ("fixed execution to data": each block always updates its
// own slab): a cluster barrier (FED), or (RELAXED) each block publishing its step count to its
// two x neighbours and waiting only for theirs.  x-halo columns are kept fresh by pushing
// boundary results into the neighbour blocks' shared memory (st.shared::cluster, DSMEM) in the
// step that computes them.
//
// Work per thread: G groups (level s, rows y0 and y0+1, VX consecutive columns), owned for the
// whole launch, so the two rows' z windows stay in registers across steps (register-rotated z
// columns): per step and plane a group loads one new z plane per row, 2R rows of y neighbours
// shared by both rows and 2R x neighbours per row, and stores one vector per row.
//
// Data movement: every thread stages elements with cp.async, MWD_PREFETCH steps ahead (a group
// committed at step k is waited for before the barrier that ends step k+PD-1), and writes back
// with plain stores; a plane is written back once the tile's top level has passed it, only rows
// of the diamond's projection, only buffers the tile updated in that row.  The ring holds
// MWD_PLAIN_SLACK*nf planes more than the wavefront needs, so no slot is restaged while a thread
// that has not yet passed the previous step's barrier still writes back from it.  This is the
// path for any layout; 16-byte aligned layouts use the vector kernel of mwd_vec.cuh.
#pragma once
#include "internal.h"
#include "stencil.cuh"

namespace girih {

// Accessor of one point of a row pair handled as VX consecutive columns.  ROW (0: row y0, 1: row
// y0+1) and I (column within the vector) are compile-time after unrolling, so every access below
// resolves to a register:
//   w      this row's z window, w[(R + dz)*VX + i]          (centre plane dz = 0)
//   other  the other row's window (its centre is this row's y neighbour at distance 1)
//   ylo    rows y0-R .. y0-1, ylo[j*VX + i] = row y0-R+j    yhi  rows y0+2 .. y0+1+R
//   xl     this row's x line: R columns left of the vector, the vector, R columns right
template <int S, typename T, int VX, int ROW, int I>
struct VecAcc {
  static constexpr int R = Traits<S>::R;
  const T* w;
  const T* other;
  const T* ylo;
  const T* yhi;
  const T* xl;
  T uc;
  const T* coef;     // coefficient grid 0 at this point (variable stencils)
  int64_t gs;        // grid stride
  __device__ __forceinline__ T c() const { return w[R * VX + I]; }
  __device__ __forceinline__ T x(int d) const { return xl[R + I + d]; }
  __device__ __forceinline__ T z(int d) const { return w[(R + d) * VX + I]; }
  __device__ __forceinline__ T y(int d) const {
    if (ROW == 0) return d < 0 ? ylo[(R + d) * VX + I] : (d == 1 ? other[R * VX + I] : yhi[(d - 2) * VX + I]);
    return d > 0 ? yhi[(d - 1) * VX + I] : (d == -1 ? other[R * VX + I] : ylo[(R + 1 + d) * VX + I]);
  }
  __device__ __forceinline__ T u() const { return uc; }
  __device__ __forceinline__ T k(int g) const { return __ldg(coef + g * gs); }
};

// VX consecutive elements from shared memory (one 16-byte access when VX*sizeof(T) == 16).
template <typename T, int VX>
__device__ __forceinline__ void lds_vec(const T* p, T* out) {
  if constexpr (VX * sizeof(T) == 16) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2*>(p);
      out[0] = v.x; out[1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < VX; ++i) out[i] = p[i];
  }
}
template <typename T, int VX>
__device__ __forceinline__ void sts_vec(T* p, const T* v) {
  if constexpr (VX * sizeof(T) == 16) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
#pragma unroll
    for (int i = 0; i < VX; ++i) p[i] = v[i];
  }
}

// Columns per thread of the element kernel: whole 16-byte vectors, except the 25-point FP64
// tiles (register budget).
template <int S, typename T>
constexpr int mwd_vx() {
  return (Traits<S>::R == 4 && sizeof(T) == 8) ? 1 : (int)(16 / sizeof(T));
}
// Launch-bound divisor for the register growth of vector groups.
template <int S, typename T>
constexpr int mwd_lbf() {
  return mwd_vx<S, T>() == 1 ? 1 : (Traits<S>::R == 1 ? 2 : 4);
}

__device__ __forceinline__ int lev_lo_of(int a, int b, int dw, int R, int t) {
  return max(a * dw - R * t, b * dw + R * t);
}
__device__ __forceinline__ int lev_hi_of(int a, int b, int dw, int R, int t) {
  return min((a + 1) * dw - R * t, (b + 1) * dw + R * t);
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Named barrier 1 of the block (barrier 0 is __syncthreads): arrive without waiting, or wait for
// all `n` threads to have arrived.
__device__ __forceinline__ void named_bar_arrive(int n) { asm volatile("bar.arrive 1, %0;" ::"r"(n) : "memory"); }
__device__ __forceinline__ void named_bar_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
__device__ __forceinline__ void fence_acq_rel_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_cluster_u32(const int* p) {
  uint32_t v;
  asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}

// ---- bulk-copy (TMA) and mbarrier helpers ---------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(ok)
               : "r"(smem_addr(m)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bound on one mbarrier wait, in nanoseconds of the global timer: a staged plane that has not
// arrived after this long sets GIRIH_ETIMEOUT in the error word and the kernel carries on.
constexpr uint64_t kMbarWaitNs = 2000000000ull;

// RELAXED hand-off: wait until the progress counters of the block's existing x neighbours
// (prog[0] left, prog[1] right, written by them with release semantics) reach `need`, for at
// most limit_ns of the global timer.  On timeout sets GIRIH_ETIMEOUT in *err and returns false.
__device__ __forceinline__ bool wait_counts(const int* prog, bool left, bool right, uint32_t need,
                                            uint64_t limit_ns, int* err) {
  const uint64_t t0 = global_ns();
  while ((left && ld_acquire_cluster_u32(&prog[0]) < need) || (right && ld_acquire_cluster_u32(&prog[1]) < need)) {
    if (global_ns() - t0 > limit_ns) {
      atomicOr(err, GIRIH_ETIMEOUT);
      return false;
    }
  }
  return true;
}

template <int N>
__device__ __forceinline__ void bulk_wait_read_n() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// The VX point updates of both rows of a group.  Columns I >= nv lie past the slab's end: their
// results are discarded, and their coefficient reads are redirected to column 0 (in bounds).
template <int S, typename T, int VX, int I>
__device__ __forceinline__ void mwd_points_i(const T* w0, const T* w1, const T* ylo, const T* yhi, const T* xl0,
                                             const T* xl1, const T* u0, const T* u1, const T* kp, int64_t gs,
                                             int64_t ldx, int nv, bool row1, const T* cst, T* r0, T* r1) {
  if constexpr (I < VX) {
    const T* k0 = (Traits<S>::NCOEF > 0 && I < nv) ? kp + I : kp;
    VecAcc<S, T, VX, 0, I> a0{w0, w1, ylo, yhi, xl0, Traits<S>::ORDER2 ? u0[I] : T(0), k0, gs};
    r0[I] = point_update<S, T>(a0, cst);
    if (row1) {
      VecAcc<S, T, VX, 1, I> a1{w1, w0, ylo, yhi, xl1, Traits<S>::ORDER2 ? u1[I] : T(0), k0 + ldx, gs};
      r1[I] = point_update<S, T>(a1, cst);
    }
    mwd_points_i<S, T, VX, I + 1>(w0, w1, ylo, yhi, xl0, xl1, u0, u1, kp, gs, ldx, nv, row1, cst, r0, r1);
  }
}
template <int S, typename T, int VX>
__device__ __forceinline__ void mwd_points(const T* w0, const T* w1, const T* ylo, const T* yhi, const T* xl0,
                                           const T* xl1, const T* u0, const T* u1, const T* kp, int64_t gs,
                                           int64_t ldx, int nv, bool row1, const T* cst, T* r0, T* r1) {
  mwd_points_i<S, T, VX, 0>(w0, w1, ylo, yhi, xl0, xl1, u0, u1, kp, gs, ldx, nv, row1, cst, r0, r1);
}

template <int S, typename T, int G>
__global__ void __launch_bounds__(1024 / (G * mwd_lbf<S, T>())) mwd_fed_kernel(const MwdArgs A) {
  constexpr int R = Traits<S>::R;
  constexpr int NC = Traits<S>::NCOEF;
  constexpr int PD = MWD_PREFETCH;
  constexpr int A16 = 16 / (int)sizeof(T);  // elements per 16 bytes
  constexpr int VX = mwd_vx<S, T>();         // columns per thread
  constexpr int OFF = VX == 1 ? R : A16;     // shared column of the slab's first column
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, nf = A.nf, K = A.K;
  const int pe = YW * XT;
  const int be = NZ * pe;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + (((size_t)2 * be * sizeof(T) + 15) / 16) * 16);
  int* lev_lo = reinterpret_cast<int*>(mbar + NZ);
  int* lev_w = lev_lo + A.H;
  int* lev_pp = lev_w + A.H;  // prefix count of row pairs per level
  int* row_mask = lev_pp + A.H + 1;
  int* prog = row_mask + A.YW;  // RELAXED: steps completed by the left [0] and right [1] neighbour

  const int nx = (int)A.g.nx, ny = (int)A.g.ny, nz = (int)A.g.nz;
  const int64_t ldx = A.g.ldx;
  const int64_t gplane = A.g.sy * A.g.ldx;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const int tile = blockIdx.x / C;
  const int dw = A.dw, rho = A.rho;
  const int a = A.a_min + tile, b = a - rho;
  const int P0 = a * dw - rho * (dw / 2);  // first y of the diamond's projection
  const int Y0 = P0 - R;                   // y of shared row 0
  const int x0 = rank * XW;
  const int xw = min(XW, nx - x0);         // this block's slab width (<= 0: idle block)
  const int Hh = A.H / 2;
  const int tb = max((rho - 1) * Hh + 1, 0);
  const int te = min((rho + 1) * Hh - 1, A.T - 1);
  if (tb > te) return;  // the whole cluster sees the same (tb, te): no barrier is skipped unevenly
  const int nlev = te - tb + 1, smax = nlev - 1;
  const int NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;

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
    prog[0] = prog[1] = 0;
  }
  for (int yy = tid; yy < YW; yy += NT) {
    const int y = Y0 + yy;
    int m = 0;
    if (y >= 0 && y < ny && y >= P0 && y < P0 + dw) {
      int cnt = 0, par = 0;
      for (int s = 0; s < nlev; ++s) {
        const int t = tb + s;
        if (y >= lev_lo_of(a, b, dw, R, t) && y < lev_hi_of(a, b, dw, R, t)) {
          ++cnt;
          par = (t + 1) & 1;
        }
      }
      m = (cnt >= 2) ? 3 : (cnt == 1 ? (1 << par) : 0);
    }
    row_mask[yy] = m;
  }
  __syncthreads();  // level tables ready

  const T* __restrict__ gb0 = static_cast<const T*>(A.buf0);
  const T* __restrict__ gb1 = static_cast<const T*>(A.buf1);
  T* go0 = static_cast<T*>(A.buf0);
  T* go1 = static_cast<T*>(A.buf1);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = sizeof(T) == 8 ? static_cast<T>(A.c[i]) : static_cast<T>(A.cf[i]);
  const int64_t gstride = A.g.gstride;

  // ---- this thread's groups (computing threads only): a group is a row pair (level s, rows y0
  // and y0+1) times VX consecutive columns, owned for the whole launch.  Per group: ring offsets
  // of (row y0, first column) in the level-t and level-t+1 buffers, current plane z and its ring
  // slot (both advance by nf per step), coefficient pointer, valid columns of the vector (ragged
  // slab tail), flags (valid, second row, push left, push right).
  int gzb_[G], gsl_[G], gvo_[G], guo_[G], gflags_[G], gnv_[G], gx_[G];
  const T* gk_[G];
  const int npairs = lev_pp[nlev];
  const int nvec = XW / VX;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int id = tid + g * NT;
    const int pr = id / nvec, xl = (id - pr * nvec) * VX;
    const bool valid = (pr < npairs) && (xl < xw);
    int s = 0;
    if (valid)
      while (lev_pp[s + 1] <= pr) ++s;
    const int y0 = valid ? lev_lo[s] + 2 * (pr - lev_pp[s]) : 0;
    const int t = tb + s;
    const int col = (y0 - Y0) * XT + xl + OFF;
    gvo_[g] = (t & 1) * be + col;
    guo_[g] = ((t & 1) ^ 1) * be + col;
    gzb_[g] = -s * K;
    const int sl = (-s * K + R) % NZ;
    gsl_[g] = sl < 0 ? sl + NZ : sl;
    gnv_[g] = min(VX, xw - xl);
    gx_[g] = xl;
    const bool row1 = valid && (y0 + 1 < lev_lo[s] + lev_w[s]);
    gflags_[g] = (valid ? 1 : 0) | (row1 ? 2 : 0) | ((C > 1 && xl < R && rank > 0) ? 4 : 0) |
                 ((C > 1 && xl + VX > XW - R && rank < C - 1) ? 8 : 0);
    gk_[g] = NC ? static_cast<const T*>(A.coef) + (int64_t)(-s * K + R) * gplane + (int64_t)(y0 + R) * ldx +
                      (x0 + xl + R)
                : nullptr;
  }
  T win[G][2][(2 * R + 1) * VX];

  // ---- staging geometry: rows y in [Y0, Y0+YW) clipped to the padded grid, columns from padded
  // x0 (interior x0 - R)
  const int ylo = max(Y0, -R), yhi = min(Y0 + YW, ny + R);
  const int nrow = max(yhi - ylo, 0);
  const int ncol = (xw > 0) ? xw + 2 * R : 0;
  int lz = -R, lsl = 0;                                  // next plane to stage and its slot
  int wz = -smax * K, wsl = ((R - smax * K) % NZ + NZ) % NZ;  // next plane to write back

  auto plain_stage = [&](int z, int slot) {
    if (z < -R || z >= nz + R) return;
    const int64_t gz = (int64_t)(z + R) * gplane;
    for (int rr = warp; rr < 2 * nrow; rr += nwarps) {
      const int p = rr >= nrow;
      const int y = ylo + rr - p * nrow;
      const T* src = (p ? gb1 : gb0) + gz + (int64_t)(y + R) * ldx + x0;
      T* dst = sm + p * be + slot * pe + (y - Y0) * XT + (OFF - R);
      for (int xx = lane; xx < ncol; xx += 32) cp_async(dst + xx, src + xx);
    }
  };
  auto plain_write = [&](int z, int slot) {
    if (z < 0 || z >= nz) return;
    const int64_t gz = (int64_t)(z + R) * gplane;
    for (int yy = warp; yy < YW; yy += nwarps) {
      const int m = row_mask[yy];
      if (m == 0) continue;
      const int64_t go = gz + (int64_t)(Y0 + yy + R) * ldx + (x0 + R);
      const T* src = sm + slot * pe + yy * XT + OFF;
      for (int xl = lane; xl < xw; xl += 32) {
        if (m & 1) go0[go + xl] = src[xl];
        if (m & 2) go1[go + xl] = src[be + xl];
      }
    }
  };

  // ---- prologue: planes of the first PD steps --------------------------------------------------
  if (xw > 0)
    for (; lz < PD * nf + R; ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) plain_stage(lz, lsl);
  cp_async_commit();
  cp_async_wait_group<0>();
  if (C > 1) cluster_barrier();
  else __syncthreads();

  const uint32_t sm_base = smem_addr(sm);
  const uint32_t left_base = (C > 1 && rank > 0) ? map_to_rank(sm_base, rank - 1) : 0u;
  const uint32_t right_base = (C > 1 && rank < C - 1) ? map_to_rank(sm_base, rank + 1) : 0u;
  const bool relaxed = C > 1 && A.relaxed;
  const uint32_t prog_base = smem_addr(prog);

  const int W = (nz + smax * K + nf - 1) / nf;
  for (int w = 0; w < W; ++w) {
    // ---- compute: this thread's groups at the planes of step w ----
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int fl = gflags_[g];
      int z = gzb_[g], sl = gsl_[g];
      const T* kp = gk_[g];
      if ((fl & 1) && z + nf > 0 && z < nz) {
        for (int f = 0; f < nf; ++f) {
          if (z >= 0 && z < nz) {
            const T* Vb = sm + gvo_[g];
            if (z == 0) {  // first plane of this level: fill the whole window
#pragma unroll
              for (int d = -R; d <= R; ++d) {
                int sd = sl + d;
                sd = sd < 0 ? sd + NZ : (sd >= NZ ? sd - NZ : sd);
                lds_vec<T, VX>(Vb + sd * pe, &win[g][0][(R + d) * VX]);
                lds_vec<T, VX>(Vb + sd * pe + XT, &win[g][1][(R + d) * VX]);
              }
            } else {  // slide the window up by one plane
              const int sd = (sl + R >= NZ) ? sl + R - NZ : sl + R;
#pragma unroll
              for (int d = 0; d < 2 * R * VX; ++d) {
                win[g][0][d] = win[g][0][d + VX];
                win[g][1][d] = win[g][1][d + VX];
              }
              lds_vec<T, VX>(Vb + sd * pe, &win[g][0][2 * R * VX]);
              lds_vec<T, VX>(Vb + sd * pe + XT, &win[g][1][2 * R * VX]);
            }
            const bool row1 = fl & 2;
            const T* P = Vb + sl * pe;  // (row y0, first column) at plane z
            T ylo[R * VX], yhi[R * VX], xl0[VX + 2 * R], xl1[VX + 2 * R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
              lds_vec<T, VX>(P + (j - R) * XT, &ylo[j * VX]);
              // row y0+1+R can lie one row past the tile when the second row is not updated
              if (j < R - 1 || row1) lds_vec<T, VX>(P + (2 + j) * XT, &yhi[j * VX]);
              else {
#pragma unroll
                for (int i = 0; i < VX; ++i) yhi[j * VX + i] = T(0);
              }
            }
#pragma unroll
            for (int d = 1; d <= R; ++d) {  // x lines: R columns each side from the ring
              xl0[R - d] = P[-d];
              xl0[R + VX - 1 + d] = P[VX - 1 + d];
              xl1[R - d] = P[XT - d];
              xl1[R + VX - 1 + d] = P[XT + VX - 1 + d];
            }
#pragma unroll
            for (int i = 0; i < VX; ++i) {
              xl0[R + i] = win[g][0][R * VX + i];
              xl1[R + i] = win[g][1][R * VX + i];
            }
            T* Ub = sm + guo_[g] + sl * pe;
            T r0[VX], r1[VX], u0[VX], u1[VX];
            if constexpr (Traits<S>::ORDER2) {
              lds_vec<T, VX>(Ub, u0);
              if (row1) lds_vec<T, VX>(Ub + XT, u1);
            }
            const int nv = gnv_[g];
            mwd_points<S, T, VX>(win[g][0], win[g][1], ylo, yhi, xl0, xl1, u0, u1, kp, gstride, ldx, nv, row1, cst,
                                 r0, r1);
            if (nv == VX) {
              sts_vec<T, VX>(Ub, r0);
              if (row1) sts_vec<T, VX>(Ub + XT, r1);
            } else {
#pragma unroll
              for (int i = 0; i < VX; ++i)
                if (i < nv) {
                  Ub[i] = r0[i];
                  if (row1) Ub[XT + i] = r1[i];
                }
            }
            if (fl & 12) {
              const uint32_t so = (uint32_t)(guo_[g] + sl * pe) * (uint32_t)sizeof(T);
#pragma unroll
              for (int i = 0; i < VX; ++i) {
                if (i >= nv) continue;
                const uint32_t oi = so + (uint32_t)(i * (int)sizeof(T));
                const int colx = gx_[g] + i;  // slab column of lane i
                if ((fl & 4) && colx < R) {  // my left edge is the left neighbour's right halo
                  st_cluster(left_base + oi + (uint32_t)(XW * (int)sizeof(T)), r0[i]);
                  if (row1) st_cluster(left_base + oi + (uint32_t)((XT + XW) * (int)sizeof(T)), r1[i]);
                }
                if ((fl & 8) && colx >= XW - R) {  // my right edge is the right neighbour's left halo
                  st_cluster(right_base + oi - (uint32_t)(XW * (int)sizeof(T)), r0[i]);
                  if (row1) st_cluster(right_base + oi + (uint32_t)((XT - XW) * (int)sizeof(T)), r1[i]);
                }
              }
            }
          }
          ++z;
          sl = (sl + 1 == NZ) ? 0 : sl + 1;
          if constexpr (NC > 0) kp += gplane;
        }
      }
      gzb_[g] += nf;
      gsl_[g] = (gsl_[g] + nf >= NZ) ? gsl_[g] + nf - NZ : gsl_[g] + nf;
      if constexpr (NC > 0) gk_[g] += nf * gplane;
    }

    if (relaxed) {
      // RELAXED: no cluster-wide barrier.  Once all warps of this block have finished the step's
      // updates and pushes (named barrier 1, on which only warp 0 waits), one thread publishes
      // the step count to the two x neighbours (release at cluster scope).  The block then
      // writes back and stages, and before the next step waits only for its own neighbours'
      // counts (acquire), i.e. for the blocks whose pushes it receives and into whose shared
      // memory it pushes.  Neighbours thus stay within one step of each other, the same overlap
      // the cluster barrier allows, without waiting for the rest of the cluster.
      cp_async_wait_group<PD - 2>();  // the planes of step w+1 are complete
      if (warp == 0) {
        named_bar_sync(NT);
        if (lane == 0) {
          fence_acq_rel_cluster();
          if (rank > 0) st_cluster_u32(map_to_rank(prog_base + 4u, rank - 1), (uint32_t)(w + 1));
          if (rank < C - 1) st_cluster_u32(map_to_rank(prog_base, rank + 1), (uint32_t)(w + 1));
        }
        __syncwarp();
      } else {
        named_bar_arrive(NT);
      }
      if (xw > 0) {
        if (w > 0)
          for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) plain_write(wz, wsl);
        for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) plain_stage(lz, lsl);
      }
      cp_async_commit();
      if (tid == 0)  // bounded wait for both neighbours; a timeout sets the error word
        wait_counts(prog, rank > 0, rank < C - 1, (uint32_t)(w + 1), kMbarWaitNs, A.err);
      __syncthreads();
    } else {
      cp_async_wait_group<PD - 2>();  // the planes of step w+1 are complete
      if (C > 1) cluster_arrive_release();
      else __syncthreads();  // a single block needs no second barrier
      if (xw > 0) {
        if (w > 0)
          for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) plain_write(wz, wsl);
        for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) plain_stage(lz, lsl);
      }
      cp_async_commit();
      if (C > 1) cluster_wait_acquire();
    }
  }
  // ---- epilogue: planes the top level finished in the last step ----
  cp_async_wait_group<0>();
  if (xw > 0)
    for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) plain_write(wz, wsl);
}

}  // namespace girih
