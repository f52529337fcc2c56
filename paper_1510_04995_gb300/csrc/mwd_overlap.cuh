// Wavefront-diamond sweep on overlapped x slabs (variant OVERLAP_PERSISTENT): the tiling,
// wavefront, persistent FIFO schedule and warp roles of RELAXED_PERSISTENT (mwd_async.cuh), with
// the per-step halo exchange between the blocks of a cluster replaced by redundant computation.
//
// Slabs.  A tile of H-1 levels (smax = H-2) has its blocks split x into slabs as before, but a
// block stages its slab plus HM >= (smax+1) R columns on each side (rounded up to 16 bytes) and
// updates level s over its slab widened by (smax - s) R columns per side: level s reads level s-1
// only inside the columns level s-1 updated, and the top level covers exactly the slab.  The
// widened columns repeat work a neighbour does for its own slab (bit for bit the same, since every
// point goes through point_update); nothing crosses between blocks inside a step, so a wavefront
// step waits for the block's own results only.  The redundant columns cost (sum over levels of
// 2 (smax - s) R rounded to vectors) / slab width extra updates: about 13 % for FP32 diamonds of
// width 8 on 68-column slabs, 2-5 % for FP64 diamonds of width 4.
//
// The one cross-block hazard left is write-after-read: a block stores the final values of its own
// slab to global memory in place, while a neighbour reads those columns, as its widened halo,
// through its staging copies of the same planes.  Each block therefore publishes to its two
// neighbours how many of its wavefront steps have landed in shared memory (a progress word in the
// neighbour's shared memory, stored once the staging copies are seen complete), and before step w
// the mover checks
// that both neighbours have staged every plane the block stores final values to in step w.  Final
// values appear only from the first level that level s+2 no longer covers (sf), so the check needs
// the neighbours' staging of step w - sf K - R: with the staging lead L the blocks may drift apart
// by L + sf K steps before one waits, and the check is off the critical path in practice.  A block
// that is ahead waits for one that is behind, never the reverse, so the cluster cannot deadlock.
//
// Warp roles: the computing warps, then a staging warp (issues the tensor copies of step w+L once
// step w-1 is done) and a waiting warp (waits for the copies of step w+2 to land, publishes,
// checks the neighbours, then releases step w+1), so that neither the copies' issue latency nor
// the progress exchange sits between two steps of the computing warps.  Barriers: FULL(w) (ids
// 1-2): computing warps and the waiting warp wait, the staging warp arrives once it has seen
// step w-2 done; DONE(w) (ids 3-4): computing warps arrive, the staging warp waits.
//
// Tasks (level s, row pair, 16-byte vector) run over the level's widened vector range, pair-major;
// consecutive lanes hold consecutive vectors of a pair, so a task takes its x neighbours from the
// neighbouring lanes (shuffles) and reads shared memory only at the ends of a pair's run and of
// the warp.  Partial vectors occur only at the grid's x boundary.
#pragma once
#include "mwd_async.cuh"

namespace girih {

__device__ __forceinline__ uint32_t ld_relaxed_cluster_u32(const int* p) {
  uint32_t v;
  asm volatile("ld.relaxed.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
// Bounded wait of a warp until the progress words of the block's existing x neighbours reach
// `need`; a timeout sets GIRIH_ETIMEOUT.  The stores of final values that this wait guards are made
// after it in program order and after a block barrier, and no store is performed speculatively.
__device__ __forceinline__ void wait_progress(const int* prog, bool left, bool right, uint32_t need, int* err) {
  auto behind = [&]() {
    return (left && ld_relaxed_cluster_u32(&prog[0]) < need) || (right && ld_relaxed_cluster_u32(&prog[1]) < need);
  };
  if (behind()) {
    const uint64_t t0 = global_ns();
    while (behind()) {
      if (global_ns() - t0 > kMbarWaitNs) {
        atomicOr(err, GIRIH_ETIMEOUT);
        break;
      }
    }
  }
  __syncwarp();
}

// One tile (diamond (a, a - rho), this block's widened x slab), or its z segment seg, from
// staging to write-back.  gstep: wavefront steps the block has run in earlier items of this
// launch (the load mbarriers serve global steps modulo kLoadBars; progress words count global
// steps).
//
// Segments (ZS; Sect. 8's parallelepiped split of the extruded diamond): segment j runs the
// tile's wavefront steps [j zseg, (j+1) zseg) (the last one to the tile's end), every level
// advancing through the same steps.  Its first staging brings in every plane the levels read at
// its first step (those of the earlier segment come from global memory), and a segment other
// than the last stores, besides the final values, the values of its last B steps, which the next
// segment reads: level s+1 reads level s R planes below its own, K + R steps back, and the
// second-order update level s-2 at the centre, 2K steps back (B = K + R or 2K).
template <int S, typename T, int G, bool ZS>
__device__ __forceinline__ void mwd_ovl_tile(const MwdArgs& A, const int rho, const int a, const int seg,
                                             int& gstep) {
  static_assert((Traits<S>::R == 1 && !Traits<S>::ORDER2 || Traits<S>::R == 4) && !Traits<S>::BOX,
                "radius-1 first-order or radius-4 stencils");
  constexpr int R = Traits<S>::R;
  constexpr int NC = Traits<S>::NCOEF;
  // columns per task: one 16-byte vector (radius-1 FP32 and the FP64 variable-coefficient
  // stencil), one column (radius-1 FP64 without coefficient grids: twice the tasks and warps for
  // a sweep bound by the FP64 pipe, which needs many independent FMAs in flight), 8 bytes
  // (radius-4 FP32) or one column (radius-4 FP64), whose 2R+1 planes per row are read from the
  // ring every step
  constexpr int VX = R == 1 ? ((sizeof(T) == 8 && NC == 0) ? 1 : 16 / (int)sizeof(T)) : (sizeof(T) == 4 ? 2 : 1);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, K = A.K;
  const int HM = A.HMO;  // staged columns on each side of the slab (a multiple of VX)
  const int L = A.lead;
  const int pe = A.PE;
  const int be = NZ * pe;
  const int ring = be;
  uint64_t* lb = reinterpret_cast<uint64_t*>(smem_raw + (((size_t)2 * be * sizeof(T) + 15) / 16) * 16);
  int* prog = reinterpret_cast<int*>(lb + kLoadBars);  // [0] left neighbour's progress, [1] right's
  int* lev_lo = prog + 4;
  int* lev_w = lev_lo + A.H;
  int* lev_f = lev_w + A.H;   // first vector of the level's widened range (shared-memory column / VX)
  int* lev_nv = lev_f + A.H;  // vectors in that range
  int* lev_tp = lev_nv + A.H;  // tasks of the levels below (H + 1 entries)
  int* tile_sf = lev_tp + A.H + 1;  // first level with final values
  int* tile_b0 = tile_sf + 1;       // first step of the band (read per step: kept out of registers)

  const int nx = (int)A.g.nx, ny = (int)A.g.ny, nz = (int)A.g.nz;
  const int ldx = (int)A.g.ldx;
  const int64_t gplane = A.g.sy * A.g.ldx;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const int dw = A.dw;
  const int b = a - rho;
  const int P0 = a * dw - rho * (dw / 2);
  const int Y0 = P0 - R;
  const int pc0 = rank * XW;      // padded column of the slab's first column
  const int sc0 = pc0 - HM;       // padded column of shared column 0
  const int cl = R - sc0;         // shared column of interior x = 0
  const int ch = nx + R - sc0;    // of interior x = nx (exclusive end)
  const int Hh = A.H / 2;
  const int tb = max((rho - 1) * Hh + 1, 0);
  const int te = min((rho + 1) * Hh - 1, A.T - 1);
  if (tb > te) return;  // uniform over the cluster
  const int nlev = te - tb + 1, smax = nlev - 1;
  const int NT = blockDim.x, tid = threadIdx.x;
  const int NTc = NT - kOvlMovers;
  const bool mover = tid >= NTc;
  const bool stager = mover && tid < NTc + 32;
  const int NF = NTc + kOvlMovers, ND = NTc + 32;  // threads of the FULL and DONE barriers
  const int lane = tid & 31;
  const uint32_t lb0 = smem_addr(&lb[0]);
  const int g0 = gstep;
  // the item's steps [ws, ws + W) of the tile's nz + smax K
  const bool last_seg = !ZS || seg + 1 >= A.nseg;
  const int ws = ZS ? seg * A.zseg : 0;
  const int W = last_seg ? nz + smax * K - ws : A.zseg;
  // from step band0 on, every value of the block's own slab is stored (all but the last segment)
  const int band0 = last_seg ? W : max(W - (Traits<S>::ORDER2 ? 2 * K : K + R), 0);
  gstep += W;

  // a row's value of level t+1 is final in the tile unless level t+2 also updates the row
  auto covers = [&](int y, int tt) {
    return tt <= te && y >= max(lev_lo_of(a, b, dw, R, tt), 0) && y < min(lev_hi_of(a, b, dw, R, tt), ny);
  };
  if (tid == 0) {
    int acc = 0, sf = nlev;
    for (int s = 0; s < nlev; ++s) {
      const int t = tb + s;
      const int lo = max(lev_lo_of(a, b, dw, R, t), 0);
      const int hi = min(lev_hi_of(a, b, dw, R, t), ny);
      const int e = (smax - s) * R;
      const int c0 = max(HM - e, cl), c1 = min(HM + XW + e, ch);
      const int f = c0 / VX, nv = c1 > c0 ? (c1 + VX - 1) / VX - f : 0;
      const int w = max(hi - lo, 0);
      lev_lo[s] = lo;
      lev_w[s] = w;
      lev_f[s] = f;
      lev_nv[s] = nv;
      lev_tp[s] = acc;
      acc += (w + 1) / 2 * nv;
      if (sf == nlev && w > 0 && (!covers(lo, t + 2) || !covers(hi - 1, t + 2))) sf = s;
    }
    lev_tp[nlev] = acc;
    *tile_sf = sf;
    *tile_b0 = band0;
  }
  __syncthreads();
  const int sf = *tile_sf;

  // ---- mover: staging copies of item step j (for step 0 planes ws - smax K - R .. ws + R,
  //      from -R at least; plane ws + j + R for step j >= 1), both buffers, completing on load
  //      mbarrier (g0 + j) mod kLoadBars ----
  const uint32_t box_bytes = (uint32_t)(YW * XT * (int)sizeof(T));
  // planes are staged in increasing z, so the ring slot of the next one ((z + R) mod NZ)
  // advances by one per plane (kept by the staging lane)
  const int zfirst = max(ws - smax * K, 0) - R;
  int next_slot = (zfirst + R) % NZ;
  auto stage_step = [&](int j) {
    const int z0 = j == 0 ? zfirst : ws + j + R, z1 = min(ws + j + R, nz + R - 1);
    if (lane == 0) {
      uint64_t* m = &lb[(g0 + j) & (kLoadBars - 1)];
      mbar_expect_tx(m, (uint32_t)(z1 >= z0 ? z1 - z0 + 1 : 0) * 2u * box_bytes);
      for (int z = z0; z <= z1; ++z) {
        tma_load_3d(sm + next_slot * pe, &A.tm[0], sc0, Y0 + R, z + R, m);
        tma_load_3d(sm + be + next_slot * pe, &A.tm[1], sc0, Y0 + R, z + R, m);
        next_slot = next_slot + 1 == NZ ? 0 : next_slot + 1;
      }
    }
    __syncwarp();
  };
  auto wait_step = [&](int j) {
    const int gs = g0 + j;
    warp_wait_phase(lb0 + (uint32_t)((gs & (kLoadBars - 1)) * 8), (uint32_t)((gs / kLoadBars) & 1), A.err);
  };
  const bool has_l = C > 1 && rank > 0, has_r = C > 1 && rank < C - 1;
  const uint32_t prog_base = smem_addr(prog);
  // the neighbours' progress words this block writes: slot 1 of the left one, slot 0 of the right
  const uint32_t pub_l = has_l ? map_to_rank(prog_base + 4u, (uint32_t)(rank - 1)) : 0u;
  const uint32_t pub_r = has_r ? map_to_rank(prog_base, (uint32_t)(rank + 1)) : 0u;
  // the staging of tile steps 0 .. j has landed: tell the neighbours (a count of steps over the
  // launch).  A relaxed store with no fence: it is issued only after the acquiring wait on the
  // load mbarrier has seen the staging copies complete, so their reads of global memory are done
  // before the count can be observed, and a neighbour stores to those columns only after
  // observing it (a release fence here would wait for the block's outstanding global stores of
  // final values on every step).
  auto publish = [&](int j) {
    if (lane == 0) {
      if (has_l) st_cluster_u32(pub_l, (uint32_t)(g0 + j + 1));
      if (has_r) st_cluster_u32(pub_r, (uint32_t)(g0 + j + 1));
    }
    __syncwarp();
  };
  // step w stores values to planes up to ws + w - s0 K (s0 = sf, or 0 in the band); a neighbour
  // stages plane z in its item step max(z - ws - R, 0): wait until both neighbours have landed
  // that step.  The counts last read are kept, so shared memory is polled only when they do not
  // already suffice.
  uint32_t seen_l = 0, seen_r = 0;
  auto check_neighbours = [&](int w) {
    const int s0 = w >= band0 ? 0 : sf;
    if (!(has_l || has_r) || s0 >= nlev) return;
    const uint32_t need = (uint32_t)(g0 + max(w - s0 * K - R, 0) + 1);
    if ((has_l && seen_l < need) || (has_r && seen_r < need)) {
      wait_progress(prog, has_l, has_r, need, A.err);
      seen_l = ld_relaxed_cluster_u32(&prog[0]);
      seen_r = ld_relaxed_cluster_u32(&prog[1]);
    }
    __syncwarp();
  };

  // ---- computing threads: tasks over the widened level ranges, G per thread ----
  int t_in[G], t_out[G], t_z[G], t_po[G], t_fl[G], t_par[G];
  const T* t_k[G];
  T* t_g[G];
  // planes z-1, z (and z+1 once loaded) of a task's two rows, in three register slots.  With
  // ROTATE the slots are used in rotation: at step w plane z-1 is in slot w mod 3, plane z in the
  // next one, and plane z+1 is loaded into the third, so nothing moves between steps (the step
  // loop is unrolled by 3).  The variable-coefficient stencil, whose prefetched coefficients
  // fill the registers, slides the window instead (the unrolled loop spilled).
  constexpr bool ROTATE = R == 1 && NC == 0;
  T t_b[G][3][2][VX];
  // rows y0-1 and y0+2 of the task's plane and, at the ends of a run, the x neighbours from
  // shared memory.  With PRE they are loaded at the end of the previous step (that plane of
  // level t was completed by level s-1 two steps before it is used), so that after the step's
  // barrier only the plane z+1 rows are loaded before the arithmetic: 7-point constant FP32
  // 645 -> 667 GLUP/s; the red-black sweep lost 3 % and the variable-coefficient one, whose
  // prefetched coefficients already fill the registers, 23 %, so they load after the barrier.
  constexpr bool PRE = S == 0;
  T t_yh[G][2][VX], t_xs[G][4];
  // radius 4 without coefficient grids (or with the single factor grid): planes z-R .. z+R-1 of
  // the task's two rows kept in registers and slid one plane per step, so only plane z+R is read
  // from the ring; the variable-coefficient stencil's 13 grids leave no registers for it
  constexpr bool WIN = R > 1 && Traits<S>::NCOEF <= 1;
  T t_w[G][2][WIN ? 2 * R * VX : 1];
  T t_kn[G][NC > 0 ? NC : 1][NC > 0 ? 2 : 1][VX];
  if (!mover) {
    const int ntask = lev_tp[nlev];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int id = tid + g * NTc;
      const bool valid = id < ntask;
      int s = 0, pr = 0, xv = 0, loc = 0, nv = 1;
      if (valid) {
        while (lev_tp[s + 1] <= id) ++s;
        nv = lev_nv[s];
        loc = id - lev_tp[s];
        pr = loc / nv;
        xv = lev_f[s] + (loc - pr * nv);
      }
      const int xl = xv * VX;  // shared column of the vector
      const int y0 = valid ? lev_lo[s] + 2 * pr : 0;
      const int t = tb + s;
      const int ro = (y0 - Y0) * XT + xl;
      // tasks without work read a fixed cell inside the slot (the warp loads and shuffles as a
      // whole while any of its lanes has work)
      t_in[g] = valid ? (t & 1) * be + ro : XT + VX;
      t_out[g] = valid ? ((t & 1) ^ 1) * be + ro : XT + VX;
      t_z[g] = ws - s * K;
      t_po[g] = (((ws - s * K + R) % NZ + NZ) % NZ) * pe;
      const int lo = max(0, cl - xl), hi = min(VX, ch - xl);
      const bool row1 = valid && (y0 + 1 < lev_lo[s] + lev_w[s]);
      const bool own = xl >= HM && xl < HM + XW;  // the vector is in the block's own slab
      const bool fin0 = valid && own && !covers(y0, t + 2), fin1 = row1 && own && !covers(y0 + 1, t + 2);
      const int xr = loc - pr * nv;  // position of the vector in its pair's run
      const bool own_l = xr == 0 || lane == 0;
      const bool own_r = xr == nv - 1 || lane == 31;
      // bits: 0 valid, 1 second row, 4 partial vector, 5 window loaded, 6 row y0 final, 7 row
      // y0+1 final, 8.. lo, 12.. hi, 16 left neighbour from shared memory, 17 right neighbour
      // from shared memory, 18 own slab (stored in a segment's band)
      t_fl[g] = (valid ? 1 : 0) | (row1 ? 2 : 0) | ((lo != 0 || hi != VX) ? 16 : 0) | (fin0 ? 64 : 0) |
                (fin1 ? 128 : 0) | (lo << 8) | (hi << 12) | (own_l ? (1 << 16) : 0) | (own_r ? (1 << 17) : 0) |
                ((ZS && valid && own) ? (1 << 18) : 0);
      t_g[g] = static_cast<T*>(((t + 1) & 1) ? A.buf1 : A.buf0) + (int64_t)(ws - s * K + R) * gplane +
               (int64_t)(y0 + R) * ldx + (sc0 + xl);
      t_par[g] = (sc0 - R + xl + y0 + t) & 1;
      t_k[g] = NC ? static_cast<const T*>(A.coef) + (int64_t)(ws - s * K + R) * gplane + (int64_t)(y0 + R) * ldx +
                        (sc0 + xl)
                  : nullptr;
    }
  }
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = sizeof(T) == 8 ? static_cast<T>(A.c[i]) : static_cast<T>(A.cf[i]);
  const int64_t gstride = A.g.gstride;

  // ---- prologue: the staging warp requests the planes of steps 0 .. L-1; the waiting warp waits
  //      for steps 0 and 1, publishes and checks the neighbours for step 0 ----
  if (stager) {
    fence_proxy_async_global();  // global data acquired before this tile -> bulk loads
    for (int j = 0; j < L && j < W; ++j) stage_step(j);
  } else if (mover) {
    wait_step(0);
    if (W > 1) wait_step(1);
    publish(W > 1 ? 1 : 0);
    check_neighbours(0);
  }
  __syncwarp();
  __syncthreads();

  if (!mover) {
    auto step = [&](const int w, auto rot) {
      constexpr int ROT = decltype(rot)::value;  // w mod 3 (radius 1)
      __syncwarp();  // the named barriers are warp-aligned instructions
      if (w > 0) sync_full(w, NF);
      if constexpr (ZS) {
        if (w == *tile_b0) {  // the band: from here on every value of the own slab goes to global memory
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (t_fl[g] & (1 << 18)) t_fl[g] |= 64 | ((t_fl[g] & 2) ? 128 : 0);
        }
      }
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
        const bool live = (fl & 1) && z >= 0 && z < nz;
        if constexpr (R > 1) {
          // radius 4: planes z-R .. z+R of both rows, R rows above and below, R columns left and
          // right, and for the second-order stencils the level t-1 centre (the output buffer
          // before it is overwritten), all from the ring
          if (!live) continue;
          const T* Vb = sm + t_in[g];
          const T* P = Vb + po;
          const bool row1 = fl & 2;
          T* Ub = sm + t_out[g] + po;
          T w0[(2 * R + 1) * VX], w1[(2 * R + 1) * VX];
          if (!WIN || !(fl & 32)) {
            int od[2 * R + 1];  // ring offsets of planes z-R .. z+R (one add and one wrap each)
            od[R] = po;
#pragma unroll
            for (int d = 1; d <= R; ++d) {
              const int up = od[R + d - 1] + pe;
              od[R + d] = up >= ring ? up - ring : up;
              const int dn = od[R - d + 1] - pe;
              od[R - d] = dn < 0 ? dn + ring : dn;
            }
#pragma unroll
            for (int d = 0; d <= 2 * R; ++d) {
              lds_vec<T, VX>(Vb + od[d], &w0[d * VX]);
              lds_vec<T, VX>(Vb + od[d] + XT, &w1[d * VX]);
            }
            if (WIN) t_fl[g] |= 32;
          } else {
            int top = po + R * pe;  // plane z+R
            top = top >= ring ? top - ring : top;
#pragma unroll
            for (int j = 0; j < 2 * R * VX; ++j) {
              w0[j] = t_w[g][0][j];
              w1[j] = t_w[g][1][j];
            }
            lds_vec<T, VX>(Vb + top, &w0[2 * R * VX]);
            lds_vec<T, VX>(Vb + top + XT, &w1[2 * R * VX]);
          }
          if constexpr (WIN) {  // the next step's planes z+1-R .. z+R
#pragma unroll
            for (int j = 0; j < 2 * R * VX; ++j) {
              t_w[g][0][j] = w0[VX + j];
              t_w[g][1][j] = w1[VX + j];
            }
          }
          T ylo[R * VX], yhi[R * VX], xl0[VX + 2 * R], xl1[VX + 2 * R];
#pragma unroll
          for (int j = 0; j < R; ++j) {
            lds_vec<T, VX>(P + (j - R) * XT, &ylo[j * VX]);
            // without a second row, row y0+1+R may lie past the tile: read row y0+R instead
            const int yo = (j == R - 1 && !row1) ? (1 + j) * XT : (2 + j) * XT;
            lds_vec<T, VX>(P + yo, &yhi[j * VX]);
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
          const int lo = (fl >> 8) & 15, hi = (fl >> 12) & 15;
          T r0[VX], r1[VX];
          mwd_points<S, T, VX>(w0, w1, ylo, yhi, xl0, xl1, u0, u1, kp, gstride, ldx, hi, true, cst, r0, r1);
          if (!(fl & 16)) {
            sts_vec<T, VX>(Ub, r0);
            if (row1) sts_vec<T, VX>(Ub + XT, r1);
            if (fl & 64) sts_vec<T, VX>(gp, r0);  // final values of the own slab go to global memory
            if (fl & 128) sts_vec<T, VX>(gp + ldx, r1);
          } else {
#pragma unroll
            for (int i = 0; i < VX; ++i)
              if (i >= lo && i < hi) {
                Ub[i] = r0[i];
                if (row1) Ub[XT + i] = r1[i];
                if (fl & 64) gp[i] = r0[i];
                if (fl & 128) gp[ldx + i] = r1[i];
              }
          }
        } else {
          if (!__any_sync(0xffffffffu, live)) continue;
          T(&zm)[2][VX] = t_b[g][ROT];
          T(&zc)[2][VX] = t_b[g][(ROT + 1) % 3];
          T(&zp)[2][VX] = t_b[g][(ROT + 2) % 3];
          const T* Vb = sm + t_in[g];
          const T* P = Vb + po;
          const bool row1 = fl & 2;
          // rows y0-1, y0+2 (without a second row, row y0+2 may lie past the tile: row y0+1 is
          // read instead) and the shared-memory x neighbours of the plane at Q
          auto load_side = [&](const T* Q) {
            lds_vec<T, VX>(Q - XT, t_yh[g][0]);
            lds_vec<T, VX>(Q + (row1 ? 2 * XT : XT), t_yh[g][1]);
            if (fl & (1 << 16)) {
              t_xs[g][0] = Q[-1];
              t_xs[g][1] = Q[XT - 1];
            }
            if (fl & (1 << 17)) {
              t_xs[g][2] = Q[VX];
              t_xs[g][3] = Q[XT + VX];
            }
          };
          if (live && !(fl & 32)) {  // first plane of the task: load the window (planes z-1, z)
            const int pm = (po == 0 ? ring : po) - pe;
            lds_vec<T, VX>(Vb + pm, zm[0]);
            lds_vec<T, VX>(Vb + pm + XT, zm[1]);
            lds_vec<T, VX>(P, zc[0]);
            lds_vec<T, VX>(P + XT, zc[1]);
            if (PRE) load_side(P);
            t_fl[g] |= 32;
          }
          const int pp = (po + pe == ring) ? 0 : po + pe;
          if (!PRE) load_side(P);
          T yr[4][VX], xm[2], xp[2];
          lds_vec<T, VX>(Vb + pp, zp[0]);
          lds_vec<T, VX>(Vb + pp + XT, zp[1]);
  #pragma unroll
          for (int i = 0; i < VX; ++i) {
            yr[0][i] = t_yh[g][0][i];
            yr[1][i] = zc[0][i];
            yr[2][i] = zc[1][i];
            yr[3][i] = t_yh[g][1][i];
          }
  #pragma unroll
          for (int r = 0; r < 2; ++r) {
            const T l = __shfl_up_sync(0xffffffffu, yr[1 + r][VX - 1], 1);
            const T q = __shfl_down_sync(0xffffffffu, yr[1 + r][0], 1);
            xm[r] = (fl & (1 << 16)) ? t_xs[g][r] : l;
            xp[r] = (fl & (1 << 17)) ? t_xs[g][2 + r] : q;
          }
          if (!live) continue;
          T r0[VX], r1[VX];
          if constexpr (NC > 0) {
            if (!(fl & 32)) load_coef_pair<T, VX, NC>(kp, gstride, ldx, t_kn[g]);  // first plane: not prefetched
            task_row2<S, T, VX, 0, 0>(yr, zm, zp, xm, xp, t_kn[g], cst, r0);
            task_row2<S, T, VX, 1, 0>(yr, zm, zp, xm, xp, t_kn[g], cst, r1);
            // prefetch the next plane's coefficients: consumed in the next step
            if (z + 1 < nz) load_coef_pair<T, VX, NC>(kp + gplane, gstride, ldx, t_kn[g]);
          } else {
            T kv[1][VX];
            task_row<S, T, VX, 0, 0>(yr, zm, zp, xm, xp, kv, cst, r0);
            task_row<S, T, VX, 1, 0>(yr, zm, zp, xm, xp, kv, cst, r1);
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
            if (fl & 64) sts_vec<T, VX>(gp, r0);  // final values of the own slab go to global memory
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
          if constexpr (!ROTATE) {  // slide the window one plane up
#pragma unroll
            for (int i = 0; i < VX; ++i) {
              zm[0][i] = zc[0][i];
              zm[1][i] = zc[1][i];
              zc[0][i] = zp[0][i];
              zc[1][i] = zp[1][i];
            }
          }
          if (PRE && z + 1 < nz) load_side(Vb + pp);  // the next plane's rows y0-1, y0+2 and x neighbours
        }
      }
      fence_proxy_async_shared();  // shared-memory results ordered before later bulk copies into the slots
      __syncwarp();
      arrive_done(w, ND);
    };
    using R0 = std::integral_constant<int, 0>;
    using R1 = std::integral_constant<int, 1>;
    using R2 = std::integral_constant<int, 2>;
    int w = 0;
    if constexpr (ROTATE) {
      for (; w + 2 < W; w += 3) {
        step(w, R0{});
        step(w + 1, R1{});
        step(w + 2, R2{});
      }
      if (w < W) step(w, R0{});
      if (w + 1 < W) step(w + 1, R1{});
    } else {
      for (; w < W; ++w) step(w, R0{});
    }
  } else if (stager) {
    // iteration it: step it-1 is done, so the slots of the planes first read at step it+L are
    // free (ring depth); arriving at FULL(it+1) here keeps the computing warps from running two
    // steps ahead of this warp's DONE waits
    for (int it = 0; it < W; ++it) {
      if (it > 0) {
        __syncwarp();
        sync_done(it - 1, ND);
      }
      __syncwarp();
      if (it + 1 < W) arrive_full(it + 1, NF);
      if (it + L < W) stage_step(it + L);
    }
    __syncwarp();
    if (W > 0) sync_done(W - 1, ND);
  } else {
    // iteration it (overlapping the computing warps' step it): the staging of step it+2 has
    // landed (a plane is in place two steps before use), published; the neighbours have staged
    // what step it+1 stores final values over; then FULL(it+1)
    for (int it = 0; it + 1 < W; ++it) {
      if (it + 2 < W) {
        wait_step(it + 2);
        publish(it + 2);
      }
      check_neighbours(it + 1);
      __syncwarp();
      sync_full(it + 1, NF);
    }
  }
}

// Persistent kernel: clusters take diamonds, or (ZS) z segments of diamonds, from the FIFO as in
// mwd_async_kernel (Sect. 4.2.3).
template <int S, typename T, int G, bool ZS>
__global__ void __launch_bounds__(async_max_threads(G, Traits<S>::NCOEF > 0, Traits<S>::R == 4), 1)
    mwd_ovl_kernel(const __grid_constant__ MwdArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C = A.C;
  const int rank = (C > 1) ? (int)cluster_ctarank() : 0;
  const size_t ring_bytes = (((size_t)2 * A.NZ * A.PE * sizeof(T) + 15) / 16) * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes);
  int* prog = reinterpret_cast<int*>(bars + kLoadBars);
  int* slot = prog + 2;
  // load mbarriers initialised and progress words cleared once per launch (the first cluster
  // barrier below orders both before any neighbour's write and any bulk copy)
  if (threadIdx.x == 0) {
    for (int i = 0; i < kLoadBars; ++i) mbar_init(&bars[i], 1);
    prog[0] = 0;
    prog[1] = 0;
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
    const int seg = ZS ? A.segs[it] : 0;
    // completion flag of (diamond (r, d), segment j)
    auto flag = [&](int r, int d, int j) { return A.flags + A.rows[3 * r] + (d - A.rows[3 * r + 1]) * A.nseg + j; };
    if (rank == 0 && threadIdx.x == 0 && (rho > 0 || seg > 0)) {
      // the tile's previous segment, and the parents' segments up to seg + delta: the parents'
      // level tb - 1 (this row's first input) lags this row's first level by (tb - tb_parent - 1) K
      // planes in the wavefront, and this tile reads R planes beyond its own
      const uint64_t t0 = global_ns();
      const bool gave_up = *reinterpret_cast<volatile int*>(A.err) != 0;
      auto wait_flag = [&](const int* f) {
        int v;
        for (;;) {
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
          if (v == A.epoch) break;
          if (global_ns() - t0 > kMbarWaitNs) {
            atomicOr(A.err, GIRIH_ETIMEOUT);
            break;
          }
        }
      };
      if (seg > 0 && !gave_up) wait_flag(flag(rho, a, seg - 1));
      if (rho > 0) {
        const int amin = A.rows[3 * (rho - 1) + 1], nd = A.rows[3 * (rho - 1) + 2];
        int jp = 0;
        if (ZS) {
          const int Hh = A.H / 2;
          const int lag = max((rho - 1) * Hh + 1, 0) - max((rho - 2) * Hh + 1, 0) - 1;
          jp = min(seg + (lag * A.K + Traits<S>::R + A.zseg - 1) / A.zseg, A.nseg - 1);
        }
        for (int d = a - 1; d <= a && !gave_up; ++d)
          if (d >= amin && d < amin + nd) wait_flag(flag(rho - 1, d, jp));
      }
    }
    // the item's completion flag (z segments: kept in shared memory over the tile, not in
    // registers; whole tiles: the FIFO position)
    if (ZS && rank == 0 && threadIdx.x == 0) slot[1] = (int)(flag(rho, a, seg) - A.flags);
    __syncwarp();
    cluster_barrier();
    mwd_ovl_tile<S, T, G, ZS>(A, rho, a, seg, gstep);
    __syncwarp();
    cluster_barrier();
    if (rank == 0 && threadIdx.x == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(A.flags + (ZS ? slot[1] : it)), "r"(A.epoch)
                   : "memory");
    }
  }
}

}  // namespace girih
