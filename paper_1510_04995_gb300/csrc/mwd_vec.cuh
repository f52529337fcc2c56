// Wavefront-diamond sweep, aligned-layout form (rows of 16-byte multiples, 16-byte aligned
// buffers).  Same tiling, ring, wavefront schedule and synchronisation as mwd_kernel.cuh (see
// the comment there); what differs is the data path, built so that every bulk movement is a
// 16-byte access and the per-update instruction count stays small:
//
//  * Shifted slab partition.  Block r of the cluster owns the padded columns
//    [r*XW, (r+1)*XW) (interior columns [r*XW - R, ...), the first R columns of block 0 being the
//    fixed halo), so a slab starts on a 16-byte boundary both in global memory and in its shared
//    row, which starts HM = R rounded up to 16 bytes columns before it.  Staging copies whole
//    16-byte chunks with cp.async; write-back stores whole 16-byte chunks of the owned columns
//    (block 0 rewrites the halo columns it staged, with the values it staged).
//  * No z window in registers: each update re-reads its 2R+1 planes from the ring (the ring
//    offsets of consecutive planes advance with one add and one wrap each), which on this part
//    costs fewer issue slots than sliding a register window, and frees the registers.
//  * Both rows of a row pair are always computed (reads clamped inside the tile); the second
//    row's stores are predicated, so a group's update is straight-line code.
//  * Data movement, two modes.  Plain: every thread stages 16-byte chunks with cp.async (global
//    pointers and shared offsets precomputed per thread, only its valid items visited) and
//    writes back 16-byte chunks with vector stores.  (Write-back by bulk stores from warp 0, which
//    spares the barrier's release the wait for generic stores, measured 26 % slower here: the
//    per-thread fence.proxy.async and warp 0's serial issue cost more than they saved.)  TMA
//    (FED_BULK): between the two halves of each step's cluster barrier, warp 0 moves whole rows
//    with the bulk-copy engine, global->shared completing on one mbarrier per ring slot (bounded
//    waits: a timeout sets the error word) and shared->global in bulk groups; the computing
//    threads only make their shared-memory results visible to the async proxy.  Bulk stores are
//    not generic stores, so the barrier's release does not wait for the write-back to reach
//    memory.  This mode stages three steps ahead and keeps a ring slack, so a slot is restaged
//    at least two steps after its last write-back was issued.
#pragma once
#include <type_traits>

#include "mwd_kernel.cuh"

namespace girih {

// Columns per group: a 16-byte vector for the 7-point stencils, 8 bytes (FP32) or one column
// (FP64) for the radius-4 stencils, whose 2R+1 planes per row would not fit in registers as
// whole vectors.
template <int S, typename T>
constexpr int vec_vx() {
  return Traits<S>::R == 1 ? (int)(16 / sizeof(T)) : (sizeof(T) == 4 ? 2 : 1);
}
template <int S>
constexpr int vec_lbf() {
  return (Traits<S>::R == 1 && !Traits<S>::BOX) ? 2 : 4;
}
constexpr int kVecItems = 4;  // precomputed staging / write-back items per thread

// Box-stencil accessor over a group's register block [3 planes][4 rows][VX+2 columns] (planes
// z-1..z+1, rows y0-1..y0+2, columns xl-1..xl+VX) for the point in row `row` (0 or 1) and
// column `col` of the group.
template <typename T, int VX>
struct BoxAcc {
  const T* blk;
  int row, col;
  __device__ __forceinline__ T b(int dx, int dy, int dz) const {
    return blk[((1 + dz) * 4 + 1 + row + dy) * (VX + 2) + 1 + col + dx];
  }
  __device__ __forceinline__ T c() const { return b(0, 0, 0); }
};

// One tile (diamond (a, a - rho) of row rho, this block's x slab) from staging to write-back.
template <int S, typename T, int G, bool TMA>
__device__ __forceinline__ void mwd_vec_tile(const MwdArgs& A, const int rho, const int a) {
  constexpr int R = Traits<S>::R;
  constexpr int NC = Traits<S>::NCOEF;
  constexpr int PD = TMA ? MWD_PREFETCH_BULK : MWD_PREFETCH;
  constexpr int A16 = 16 / (int)sizeof(T);
  constexpr int VX = vec_vx<S, T>();
  constexpr int HM = (R + A16 - 1) / A16 * A16;  // shared column of the slab's first column
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, nf = A.nf, K = A.K;
  const int pe = YW * XT;
  const int be = NZ * pe;
  const int ring = NZ * pe;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + (((size_t)2 * be * sizeof(T) + 15) / 16) * 16);
  int* lev_lo = reinterpret_cast<int*>(mbar + NZ);
  int* lev_w = lev_lo + A.H;
  int* lev_pp = lev_w + A.H;
  int* row_mask = lev_pp + A.H + 1;
  int* prog = row_mask + YW;

  const int nx = (int)A.g.nx, ny = (int)A.g.ny, nz = (int)A.g.nz;
  const int ldx = (int)A.g.ldx;
  const int64_t gplane = A.g.sy * A.g.ldx;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const int dw = A.dw;
  const int b = a - rho;
  const int P0 = a * dw - rho * (dw / 2);
  const int Y0 = P0 - R;
  const int pc0 = rank * XW;          // padded column of slab column 0
  const int x0 = pc0 - R;             // its interior column
  const int vlo = max(0, -x0);        // valid slab columns [vlo, vhi)
  const int vhi = min(XW, nx - x0);
  const bool active = vhi > vlo;
  const int Hh = A.H / 2;
  const int tb = max((rho - 1) * Hh + 1, 0);
  const int te = min((rho + 1) * Hh - 1, A.T - 1);
  if (tb > te) return;
  const int nlev = te - tb + 1, smax = nlev - 1;
  const int NT = blockDim.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

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
    if constexpr (TMA) {
      for (int q = 0; q < NZ; ++q) mbar_init(&mbar[q], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
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
  __syncthreads();

  T* go0 = static_cast<T*>(A.buf0);
  T* go1 = static_cast<T*>(A.buf1);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = sizeof(T) == 8 ? static_cast<T>(A.c[i]) : static_cast<T>(A.cf[i]);
  const int64_t gstride = A.g.gstride;

  // ---- groups: row pair (level s, rows y0, y0+1) x VX columns, owned for the whole launch ----
  int gin_[G], gout_[G], gzb_[G], gpo_[G], gfl_[G], glo_[G], ghi_[G], gx_[G];
  int gpar_[G];  // red-black: parity of (x + y0 + t) at the group's first column
  const T* gk_[G];
  const int npairs = lev_pp[nlev];
  const int nvec = XW / VX;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int id = tid + g * NT;
    const int pr = id / nvec, xl = (id - pr * nvec) * VX;
    const bool valid = active && pr < npairs && xl + VX > vlo && xl < vhi;
    int s = 0;
    if (valid)
      while (lev_pp[s + 1] <= pr) ++s;
    const int y0 = valid ? lev_lo[s] + 2 * (pr - lev_pp[s]) : 0;
    const int t = tb + s;
    const int ro = (y0 - Y0) * XT + HM + xl;
    gin_[g] = (t & 1) * be + ro;
    gout_[g] = ((t & 1) ^ 1) * be + ro;
    gzb_[g] = -s * K;
    const int sl = ((-s * K + R) % NZ + NZ) % NZ;
    gpo_[g] = sl * pe;
    glo_[g] = max(0, vlo - xl);
    gx_[g] = xl;
    gpar_[g] = (x0 + xl + y0 + t) & 1;
    ghi_[g] = min(VX, vhi - xl);
    const bool row1 = valid && (y0 + 1 < lev_lo[s] + lev_w[s]);
    // x-halo pushes: the slab's first R columns to the left neighbour, its last R columns to the
    // right neighbour when that one has columns (a full slab here means it does)
    gfl_[g] = (valid ? 1 : 0) | (row1 ? 2 : 0) | ((C > 1 && rank > 0 && xl < R) ? 4 : 0) |
              ((C > 1 && rank < C - 1 && vhi == XW && xl + VX > XW - R) ? 8 : 0);
    gk_[g] = NC ? static_cast<const T*>(A.coef) + (int64_t)(-s * K + R) * gplane + (int64_t)(y0 + R) * ldx +
                      (x0 + xl + R)
                : nullptr;
  }

  // ---- staging items: (buffer, row, 16-byte chunk) of a plane; offsets relative to the plane ----
  const int ylo = max(Y0, -R), yhi = min(Y0 + YW, ny + R);
  const int nrow = active ? max(yhi - ylo, 0) : 0;
  const int cb = max(pc0 - HM, 0), ce = min(pc0 + XW + HM, ldx);
  const int nch = active ? (ce - cb) / A16 : 0;
  const int nstage = 2 * nrow * nch;
  // this thread's items: global address at plane 0 (buffer included) and shared byte offset in
  // slot 0; items tid, tid + NT, ... so the valid ones are a prefix of length n_s
  const T* s_ptr[kVecItems];
  uint32_t s_off[kVecItems];
  int n_s = 0;
#pragma unroll
  for (int i = 0; i < kVecItems; ++i) {
    const int idx = tid + i * NT;
    s_ptr[i] = static_cast<const T*>(A.buf0);
    s_off[i] = 0;
    if (idx < nstage) {
      const int p = idx / (nrow * nch);
      const int rem = idx - p * nrow * nch;
      const int r = rem / nch, ch = rem - r * nch;
      const int y = ylo + r, pc = cb + ch * A16;
      s_ptr[i] = static_cast<const T*>(p ? A.buf1 : A.buf0) + (int64_t)(y + R) * ldx + pc;
      s_off[i] = (uint32_t)((p * be + (y - Y0) * XT + (pc - (pc0 - HM))) * (int)sizeof(T));
      n_s = i + 1;
    }
  }
  // ---- write-back items: (row of the diamond's projection, 16-byte chunk of the owned columns) ----
  const int wy0 = max(P0, 0), wy1 = min(P0 + dw, ny);
  const int wb = pc0, wcend = min(pc0 + XW, ldx);
  const int nchw = active ? max((wcend - wb) / A16, 0) : 0;
  const int nwb = max(wy1 - wy0, 0) * nchw;
  int w_sm[kVecItems], w_gl[kVecItems], n_w = 0;  // valid items are a prefix of length n_w
#pragma unroll
  for (int i = 0; i < kVecItems; ++i) {
    const int idx = tid + i * NT;
    w_sm[i] = 0;
    w_gl[i] = 0;
    if (idx < nwb) {
      const int r = idx / nchw, ch = idx - r * nchw;
      const int yy = wy0 + r - Y0;
      w_sm[i] = (row_mask[yy] << 28) | (yy * XT + HM + ch * A16);  // mask in bits 28-29
      w_gl[i] = (wy0 + r + R) * ldx + wb + ch * A16;
      n_w = i + 1;
    }
  }

  const char* gb0 = static_cast<const char*>(A.buf0);
  const char* gb1 = static_cast<const char*>(A.buf1);
  const uint32_t sm_u32 = smem_addr(sm);
  auto stage = [&](int z, int slot) {
    if (z < -R || z >= nz + R) return;
    const int64_t zo = (int64_t)(z + R) * gplane;
    const uint32_t dst = sm_u32 + (uint32_t)(slot * pe * (int)sizeof(T));
#pragma unroll
    for (int i = 0; i < kVecItems; ++i) {
      if (i >= n_s) break;
      cp_async16_cg_u32(dst + s_off[i], s_ptr[i] + zo);
    }
    for (int idx = tid + kVecItems * NT; idx < nstage; idx += NT) {  // tiles wider than the items
      const int p = idx / (nrow * nch);
      const int rem = idx - p * nrow * nch;
      const int r = rem / nch, ch = rem - r * nch;
      const int y = ylo + r, pc = cb + ch * A16;
      const T* src = reinterpret_cast<const T*>(p ? gb1 : gb0) + zo + (int64_t)(y + R) * ldx + pc;
      cp_async16_cg(sm + slot * pe + p * be + (y - Y0) * XT + (pc - (pc0 - HM)), src);
    }
  };

  auto write_back = [&](int z, int slot) {
    if (z < 0 || z >= nz) return;
    const int64_t zo = (int64_t)(z + R) * gplane;
    const T* src = sm + slot * pe;
#pragma unroll
    for (int i = 0; i < kVecItems; ++i) {
      if (i >= n_w) break;
      const int m = (w_sm[i] >> 28) & 3, so = w_sm[i] & 0x0fffffff;
      if (m & 1) *reinterpret_cast<V16*>(go0 + zo + w_gl[i]) = *reinterpret_cast<const V16*>(src + so);
      if (m & 2) *reinterpret_cast<V16*>(go1 + zo + w_gl[i]) = *reinterpret_cast<const V16*>(src + be + so);
    }
    for (int idx = tid + kVecItems * NT; idx < nwb; idx += NT) {
      const int r = idx / nchw, ch = idx - r * nchw;
      const int yy = wy0 + r - Y0;
      const int m = row_mask[yy], so = yy * XT + HM + ch * A16;
      const int64_t gofs = zo + (int64_t)(wy0 + r + R) * ldx + wb + ch * A16;
      if (m & 1) *reinterpret_cast<V16*>(go0 + gofs) = *reinterpret_cast<const V16*>(src + so);
      if (m & 2) *reinterpret_cast<V16*>(go1 + gofs) = *reinterpret_cast<const V16*>(src + be + so);
    }
  };

  // TMA mode (warp 0): rows of both buffers of plane z into ring slot `slot`, one mbarrier each
  const uint32_t srow_bytes = (uint32_t)(nch * 16);
  auto tma_stage = [&](int z, int slot) {
    if (z < -R || z >= nz + R) return;
    if (lane == 0) mbar_expect_tx(&mbar[slot], srow_bytes * 2u * (uint32_t)nrow);
    __syncwarp();
    const int64_t zo = (int64_t)(z + R) * gplane;
    for (int rr = lane; rr < 2 * nrow; rr += 32) {
      const int p = rr >= nrow;
      const int y = ylo + rr - p * nrow;
      bulk_load(sm + p * be + slot * pe + (y - Y0) * XT + (cb - (pc0 - HM)),
                reinterpret_cast<const T*>(p ? gb1 : gb0) + zo + (int64_t)(y + R) * ldx + cb, srow_bytes,
                &mbar[slot]);
    }
  };
  auto tma_wait = [&](int z) {  // lane 0: bounded wait for plane z; error word on timeout
    if (z < -R || z >= nz + R) return;
    if (lane == 0) {
      const int q = z + R;
      const int slot = q % NZ;
      const uint32_t parity = (uint32_t)((q / NZ) & 1);
      if (!mbar_try_wait(&mbar[slot], parity)) {
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(&mbar[slot], parity)) {
          if (global_ns() - t0 > kMbarWaitNs) {
            atomicOr(A.err, GIRIH_ETIMEOUT);
            break;
          }
        }
      }
    }
    __syncwarp();
  };
  const uint32_t wrow_bytes = (uint32_t)(nchw * 16);
  auto tma_write = [&](int z, int slot) {  // masked rows of plane z, one bulk group per call and lane
    if (z >= 0 && z < nz) {
      const int64_t zo = (int64_t)(z + R) * gplane;
      for (int yy = wy0 - Y0 + lane; yy < wy1 - Y0; yy += 32) {
        const int m = row_mask[yy];
        const int64_t go = zo + (int64_t)(Y0 + yy + R) * ldx + pc0;
        const T* src = sm + slot * pe + yy * XT + HM;
        if (m & 1) bulk_store(go0 + go, src, wrow_bytes);
        if (m & 2) bulk_store(go1 + go, src + be, wrow_bytes);
      }
    }
    bulk_commit();
  };

  int lz = -R, lsl = 0;
  int wz = -smax * K, wsl = ((R - smax * K) % NZ + NZ) % NZ;
  if constexpr (TMA) {
    if (warp == 0 && active) {
      for (; lz < PD * nf + R; ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) tma_stage(lz, lsl);
      for (int z = -R; z < PD * nf + R; ++z) tma_wait(z);
    }
    cluster_barrier();
  } else {
    for (; lz < PD * nf + R; ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) stage(lz, lsl);
    cp_async_commit();
    cp_async_wait_group<0>();
    if (C > 1) cluster_barrier();
    else __syncthreads();
  }

  const uint32_t sm_base = smem_addr(sm);
  const uint32_t left_base = (C > 1 && rank > 0) ? map_to_rank(sm_base, rank - 1) : 0u;
  const uint32_t right_base = (C > 1 && rank < C - 1) ? map_to_rank(sm_base, rank + 1) : 0u;
  const bool relaxed = !TMA && C > 1 && A.relaxed;
  const uint32_t prog_base = smem_addr(prog);

  const int W = (nz + smax * K + nf - 1) / nf;
  for (int w = 0; w < W; ++w) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int fl = gfl_[g];
      int z = gzb_[g], po = gpo_[g];
      const T* kp = gk_[g];
      if ((fl & 1) && z + nf > 0 && z < nz) {
        for (int f = 0; f < nf; ++f) {
          if (z >= 0 && z < nz) {
            // ring offsets of planes z-R .. z+R (one add and one wrap each)
            int od[2 * R + 1];
            od[R] = po;
#pragma unroll
            for (int d = 1; d <= R; ++d) {
              const int up = od[R + d - 1] + pe;
              od[R + d] = up >= ring ? up - ring : up;
              const int dn = od[R - d + 1] - pe;
              od[R - d] = dn < 0 ? dn + ring : dn;
            }
            const T* Vb = sm + gin_[g];
            const bool row1 = fl & 2;
            T* Ub = sm + gout_[g] + po;
            T r0[VX], r1[VX];
            const int lo = glo_[g], hi = ghi_[g];
            if constexpr (Traits<S>::BOX) {
              // planes z-1 .. z+1 x rows y0-1 .. y0+2 x columns xl-1 .. xl+VX around the group
              // (without a second row, row y0+2 may lie past the tile: read row y0+1 instead)
              T blk[3 * 4 * (VX + 2)];
#pragma unroll
              for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const int yo = (j == 3 && !row1) ? 2 : j;
                  const T* q = Vb + od[d] + (yo - 1) * XT;
                  T* bl = &blk[(d * 4 + j) * (VX + 2)];
                  lds_vec<T, VX>(q, bl + 1);
                  bl[0] = q[-1];
                  bl[VX + 1] = q[VX];
                }
#pragma unroll
              for (int i = 0; i < VX; ++i) {
                r0[i] = point_update<S, T>(BoxAcc<T, VX>{blk, 0, i}, cst);
                r1[i] = point_update<S, T>(BoxAcc<T, VX>{blk, 1, i}, cst);
              }
            } else {
              T w0[(2 * R + 1) * VX], w1[(2 * R + 1) * VX];
#pragma unroll
              for (int d = 0; d <= 2 * R; ++d) {
                lds_vec<T, VX>(Vb + od[d], &w0[d * VX]);
                lds_vec<T, VX>(Vb + od[d] + XT, &w1[d * VX]);
              }
              const T* P = Vb + po;
              T ylo_[R * VX], yhi_[R * VX], xl0[VX + 2 * R], xl1[VX + 2 * R];
#pragma unroll
              for (int j = 0; j < R; ++j) {
                lds_vec<T, VX>(P + (j - R) * XT, &ylo_[j * VX]);
                // without a second row, row y0+1+R may lie past the tile: read row y0+R instead
                const int yo = (j == R - 1 && !row1) ? (1 + j) * XT : (2 + j) * XT;
                lds_vec<T, VX>(P + yo, &yhi_[j * VX]);
              }
#pragma unroll
              for (int d = 1; d <= R; ++d) {
                xl0[R - d] = P[-d];
                xl0[R + VX - 1 + d] = P[VX - 1 + d];
                xl1[R - d] = P[XT - d];
                xl1[R + VX - 1 + d] = P[XT + VX - 1 + d];
              }
#pragma unroll
              for (int i = 0; i < VX; ++i) {
                xl0[R + i] = w0[R * VX + i];
                xl1[R + i] = w1[R * VX + i];
              }
              T u0[VX], u1[VX];
              if constexpr (Traits<S>::ORDER2) {
                lds_vec<T, VX>(Ub, u0);
                lds_vec<T, VX>(Ub + XT, u1);
              }
              mwd_points<S, T, VX>(w0, w1, ylo_, yhi_, xl0, xl1, u0, u1, kp, gstride, ldx, hi, true, cst, r0, r1);
              if constexpr (Traits<S>::RB) {
                // red-black: only points with (x + y + z + t) even are updated, the others keep
                // their value (row y0+1 has the other colour)
#pragma unroll
                for (int i = 0; i < VX; ++i) {
                  const bool odd0 = (gpar_[g] + i + z) & 1;
                  if (odd0) r0[i] = w0[R * VX + i];
                  else r1[i] = w1[R * VX + i];
                }
              }
            }
            if (lo == 0 && hi == VX) {
              sts_vec<T, VX>(Ub, r0);
              if (row1) sts_vec<T, VX>(Ub + XT, r1);
            } else {
#pragma unroll
              for (int i = 0; i < VX; ++i)
                if (i >= lo && i < hi) {
                  Ub[i] = r0[i];
                  if (row1) Ub[XT + i] = r1[i];
                }
            }
            if (fl & 12) {
              // lanes holding the slab's first / last R columns: [0, R) / [VX-R, VX) of the edge
              // vector when VX >= R, else every lane of the R/VX edge groups
              constexpr int NL = VX >= R ? R : VX;
              const uint32_t so = (uint32_t)(gout_[g] + po) * (uint32_t)sizeof(T);
              if (fl & 4) {
#pragma unroll
                for (int i = 0; i < NL; ++i) {
                  const uint32_t oi = so + (uint32_t)(i * (int)sizeof(T)) + (uint32_t)(XW * (int)sizeof(T));
                  st_cluster(left_base + oi, r0[i]);
                  if (row1) st_cluster(left_base + oi + (uint32_t)(XT * (int)sizeof(T)), r1[i]);
                }
              }
              if (fl & 8) {
#pragma unroll
                for (int i = VX - NL; i < VX; ++i) {
                  const uint32_t oi = so + (uint32_t)(i * (int)sizeof(T)) - (uint32_t)(XW * (int)sizeof(T));
                  st_cluster(right_base + oi, r0[i]);
                  if (row1) st_cluster(right_base + oi + (uint32_t)(XT * (int)sizeof(T)), r1[i]);
                }
              }
            }
          }
          ++z;
          po = (po + pe == ring) ? 0 : po + pe;
          if constexpr (NC > 0) kp += gplane;
        }
      }
      gzb_[g] += nf;
      {
        int p2 = gpo_[g] + nf * pe;
        gpo_[g] = p2 >= ring ? p2 - ring : p2;
      }
      if constexpr (NC > 0) gk_[g] += nf * gplane;
    }

    if constexpr (TMA) {
      fence_proxy_async();  // this step's shared-memory results become visible to bulk stores
      // the planes of step w+1 (staged PD-1 steps ago) have landed before anyone may pass this
      // step's barrier
      if (warp == 0 && active)
        for (int f = 0; f < nf; ++f) tma_wait((w + 1) * nf + R + f);
      cluster_arrive_release();
      if (warp == 0 && active) {
        // restage first: the slots of step w+PD were last written back two or more steps ago, so
        // only the previous step's nf write-back groups may still be reading shared memory
        if (nf == 1) bulk_wait_read_n<1>();
        else if (nf == 2) bulk_wait_read_n<2>();
        else if (nf == 3) bulk_wait_read_n<3>();
        else bulk_wait_read_n<4>();
        __syncwarp();
        for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) tma_stage(lz, lsl);
        for (int f = 0; f < nf; ++f) {  // planes the top level finished in step w-1 (nf groups)
          if (w > 0) {
            tma_write(wz, wsl);
            ++wz;
            wsl = (wsl + 1 == NZ) ? 0 : wsl + 1;
          } else {
            bulk_commit();
          }
        }
      }
      cluster_wait_acquire();
    } else if (relaxed) {
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
      if (w > 0)
        for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) write_back(wz, wsl);
      for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) stage(lz, lsl);
      cp_async_commit();
      if (tid == 0) wait_counts(prog, rank > 0, rank < C - 1, (uint32_t)(w + 1), kMbarWaitNs, A.err);
      __syncthreads();
    } else {
      cp_async_wait_group<PD - 2>();  // the planes of step w+1 are complete
      if (C > 1) cluster_arrive_release();
      else __syncthreads();
      if (w > 0)
        for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) write_back(wz, wsl);
      for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) stage(lz, lsl);
      cp_async_commit();
      if (C > 1) cluster_wait_acquire();
    }
  }
  if constexpr (TMA) {
    if (warp == 0 && active) {
      for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) tma_write(wz, wsl);
      bulk_wait_all();  // the shared source must outlive the copies
    }
  } else {
    cp_async_wait_group<0>();
    for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) write_back(wz, wsl);
  }
}

// The kernel: one tile per cluster per launch (one launch per diamond row), or, persistent
// (FED_PERSISTENT), every cluster of a grid that fits the device at once takes diamonds from a
// FIFO in row-major order -- the runtime of Sect. 4.2.3 -- and starts a diamond once the two
// diamonds of the previous row it depends on ((a-1, b) and (a, b+1)) have published completion.
// Their y projections cover the diamond's projection plus R rows each side, so every value the
// diamond reads is final; diamonds that are not dependencies are at least Dw/2 rows away.  The
// FIFO order is a topological order and all clusters are resident, so the waits cannot
// deadlock; each is bounded (a timeout sets GIRIH_ETIMEOUT) all the same.  Completion: after a
// cluster barrier (all blocks' write-back stores ordered at cluster scope), one thread releases
// the diamond's flag at GPU scope (fence.acq_rel.gpu); the waiting cluster acquires it.
template <int S, typename T, int G, bool TMA>
__global__ void __launch_bounds__(1024 / (G * vec_lbf<S>()), 1) mwd_vec_kernel(const MwdArgs A) {
  if (!A.persist) {
    mwd_vec_tile<S, T, G, TMA>(A, A.rho, A.a_min + (int)blockIdx.x / A.C);
    return;
  }
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C = A.C;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const size_t ring_bytes = (((size_t)2 * A.NZ * A.YW * A.XT * sizeof(T) + 15) / 16) * 16;
  int* slot = reinterpret_cast<int*>(smem_raw + ring_bytes + 8 * (size_t)A.NZ) + 3 * A.H + 1 + A.YW + 2;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const int it = atomicAdd(A.fifo, 1);
      for (int r = 0; r < C; ++r) st_cluster_u32(map_to_rank(smem_addr(slot), (uint32_t)r), (uint32_t)it);
    }
    cluster_barrier();
    const int it = *reinterpret_cast<volatile int*>(slot);
    if (it >= A.n_items) break;
    const int rho = A.items[2 * it], a = A.items[2 * it + 1];
    if (rank == 0 && threadIdx.x == 0 && rho > 0) {
      const int first = A.rows[3 * (rho - 1)], amin = A.rows[3 * (rho - 1) + 1], nd = A.rows[3 * (rho - 1) + 2];
      const uint64_t t0 = global_ns();
      // after a timeout anywhere in the sweep the result is void: stop waiting so the launch ends
      const bool gave_up = *reinterpret_cast<volatile int*>(A.err) != 0;
      for (int d = a - 1; d <= a && !gave_up; ++d) {
        if (d < amin || d >= amin + nd) continue;  // outside the grid: nothing to wait for
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
    cluster_barrier();
    mwd_vec_tile<S, T, G, TMA>(A, rho, a);
    cluster_barrier();
    if (rank == 0 && threadIdx.x == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(A.flags + it), "r"(A.epoch) : "memory");
    }
  }
}

}  // namespace girih
