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
// both buffers in shared memory: [2][NZ][YW = Dw + 2R][XT = XW + 2R].  The wavefront walks up in
// z (Sect. 2.1.1): at step w, local level s updates planes [w*nf - s*K, w*nf - s*K + nf) with the
// level skew K = R + nf, which makes every input of a step come from earlier steps, so one
// cluster barrier per step is the only synchronisation ("fixed execution to data": each block
// always updates its own slab).  x-halo columns are kept fresh by pushing boundary results into
// the neighbour blocks' shared memory (st.shared::cluster, DSMEM) before the barrier.  Planes are
// staged in with cp.async one step ahead of use; a plane is written back to HBM once the tile's
// top level has passed it (only the rows of the tile's projection that the tile updated).
#include "internal.h"
#include "stencil.cuh"

namespace girih {

// Accessor of one row of a row pair: z neighbours and the centre come from the thread's own
// register window (w[R] = centre), y neighbours from the pair's shared loads (yl), x neighbours
// and the level t-1 centre from the shared ring.
template <int S, typename T>
struct PairAcc {
  const T* w;        // window of this row, planes z-R..z+R
  const T* yv;       // y neighbours: yv[R + d] = value at row y + d (d != 0)
  const T* X;        // pointer to the centre in the level-t ring buffer
  T uc;
  const T* coef;     // coefficient grid 0 at this pair's first row and current plane
  int64_t gs, p;     // grid stride, offset of this row from coef
  __device__ __forceinline__ T c() const { return w[Traits<S>::R]; }
  __device__ __forceinline__ T x(int d) const { return X[d]; }
  __device__ __forceinline__ T y(int d) const { return yv[Traits<S>::R + d]; }
  __device__ __forceinline__ T z(int d) const { return w[Traits<S>::R + d]; }
  __device__ __forceinline__ T u() const { return uc; }
  __device__ __forceinline__ T k(int g) const { return __ldg(coef + g * gs + p); }
};

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

// G = row pairs owned per thread.  Each pair (level s, rows y0 and y0+1, column xl) is owned
// by one thread for the whole launch (fixed execution to data), which keeps the two rows'
// z windows in registers across wavefront steps: per step and plane, a pair loads 2 new z
// values, 2R rows of y neighbours shared by both rows, 2R x neighbours per row, and stores 2.
// Step w: compute; wait for this thread's staged planes of step w+1; cluster arrive (release:
// publishes the step's shared and DSMEM writes); write back the planes the top level finished
// in step w-1 and stage the planes of step w+PD (both overlap the barrier, and the write-back
// stores are not held by the release); cluster wait (acquire).  The write-back and staging may
// run while other threads already compute step w+1: the ring depth keeps those planes apart.
// A single block (C = 1) uses one __syncthreads in place of the arrive.
// All per-pair and per-plane positions advance incrementally: no division in the step loop.
template <int S, typename T, int G>
__global__ void __launch_bounds__(1024 / G) mwd_fed_kernel(const MwdArgs A) {
  constexpr int R = Traits<S>::R;
  constexpr int NC = Traits<S>::NCOEF;
  constexpr int PD = MWD_PREFETCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, nf = A.nf, K = A.K;
  const int pe = YW * XT;
  const int be = NZ * pe;
  int* lev_lo = reinterpret_cast<int*>(sm + 2 * be);
  int* lev_w = lev_lo + A.H;
  int* lev_pp = lev_w + A.H;  // prefix count of row pairs per level
  int* row_mask = lev_pp + A.H + 1;

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

  // ---- this thread's row pairs --------------------------------------------------------------
  // per pair: level s, ring offsets of row y0 in the level-t and level-t+1 buffers, current
  // plane z and its ring slot (both advance by nf per step), coefficient pointer, push flags
  int gzb_[G], gsl_[G], gvo_[G], guo_[G], gflags_[G];
  const T* gk_[G];
  const int npairs = lev_pp[nlev];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int id = tid + g * NT;
    const int pr = id / XW, xl = id - pr * XW;
    const bool valid = (pr < npairs) && (xl < xw);
    int s = 0;
    if (pr < npairs)
      while (lev_pp[s + 1] <= pr) ++s;
    const int y0 = (pr < npairs) ? lev_lo[s] + 2 * (pr - lev_pp[s]) : 0;
    const int t = tb + s;
    const int col = (y0 - Y0) * XT + xl + R;
    gvo_[g] = (t & 1) * be + col;
    guo_[g] = ((t & 1) ^ 1) * be + col;
    gzb_[g] = -s * K;
    int sl = (-s * K + R) % NZ;
    gsl_[g] = sl < 0 ? sl + NZ : sl;
    const bool row1 = (pr < npairs) && (y0 + 1 < lev_lo[s] + lev_w[s]);
    gflags_[g] = (valid ? 1 : 0) | (row1 ? 2 : 0) | ((C > 1 && xl < R && rank > 0) ? 4 : 0) |
                 ((C > 1 && xl >= XW - R && rank < C - 1) ? 8 : 0);
    gk_[g] = NC ? static_cast<const T*>(A.coef) + (int64_t)(-s * K + R) * gplane + (int64_t)(y0 + R) * ldx +
                      (x0 + xl + R)
                : nullptr;
  }
  T win[G][2][2 * R + 1];

  // ---- plane staging (cp.async) and write-back, row by row: warp k takes rows k, k+nwarps, ...
  const int ylo = max(Y0, -R), yhi = min(Y0 + YW, ny + R);
  const int nrow = max(yhi - ylo, 0);
  const int ncol = (xw > 0) ? xw + 2 * R : 0;
  // next plane to stage and its ring slot; next plane to write back and its ring slot
  int lz = -R, lsl = 0;
  int wz = -smax * K, wsl = ((R - smax * K) % NZ + NZ) % NZ;

  if (xw > 0) {
    for (; lz < PD * nf + R; ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) {
      const int64_t gz = (int64_t)(lz + R) * gplane;
      for (int rr = warp; rr < 2 * nrow; rr += nwarps) {
        const int p = rr >= nrow;
        const int y = ylo + rr - p * nrow;
        const T* src = (p ? gb1 : gb0) + gz + (int64_t)(y + R) * ldx + x0;
        T* dst = sm + p * be + lsl * pe + (y - Y0) * XT;
        for (int xx = lane; xx < ncol; xx += 32) cp_async(dst + xx, src + xx);
      }
    }
  }
  cp_async_commit();
  cp_async_wait_group<0>();
  if (C > 1) cluster_barrier();
  else __syncthreads();

  const uint32_t sm_base = smem_addr(sm);
  const uint32_t left_base = (C > 1 && rank > 0) ? map_to_rank(sm_base, rank - 1) : 0u;
  const uint32_t right_base = (C > 1 && rank < C - 1) ? map_to_rank(sm_base, rank + 1) : 0u;

  const int W = (nz + smax * K + nf - 1) / nf;
  for (int w = 0; w < W; ++w) {
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
                win[g][0][R + d] = Vb[sd * pe];
                win[g][1][R + d] = Vb[sd * pe + XT];
              }
            } else {  // slide the window up by one plane
              const int sd = (sl + R >= NZ) ? sl + R - NZ : sl + R;
#pragma unroll
              for (int d = 0; d < 2 * R; ++d) {
                win[g][0][d] = win[g][0][d + 1];
                win[g][1][d] = win[g][1][d + 1];
              }
              win[g][0][2 * R] = Vb[sd * pe];
              win[g][1][2 * R] = Vb[sd * pe + XT];
            }
            const bool row1 = fl & 2;
            const T* P = Vb + sl * pe;  // centre of row y0 at plane z
            T yv0[2 * R + 1], yv1[2 * R + 1];  // y neighbours of row y0 and row y0+1
#pragma unroll
            for (int d = 1; d <= R; ++d) {
              yv0[R - d] = P[-d * XT];
              // row y0+1+R can lie one row past the tile when the second row is not updated
              yv1[R + d] = (d < R || row1) ? P[(1 + d) * XT] : T(0);
            }
#pragma unroll
            for (int d = 1; d <= R; ++d) {
              yv0[R + d] = (d == 1) ? win[g][1][R] : yv1[R + d - 1];
              yv1[R - d] = (d == 1) ? win[g][0][R] : yv0[R - d + 1];
            }
            T* Ub = sm + guo_[g] + sl * pe;
            PairAcc<S, T> acc0{win[g][0], yv0, P, T(0), kp, gstride, 0};
            if constexpr (Traits<S>::ORDER2) acc0.uc = Ub[0];
            const T r0 = point_update<S, T>(acc0, cst);
            Ub[0] = r0;
            T r1 = T(0);
            if (row1) {
              PairAcc<S, T> acc1{win[g][1], yv1, P + XT, T(0), kp, gstride, ldx};
              if constexpr (Traits<S>::ORDER2) acc1.uc = Ub[XT];
              r1 = point_update<S, T>(acc1, cst);
              Ub[XT] = r1;
            }
            if (fl & 12) {
              const uint32_t so = (uint32_t)(guo_[g] + sl * pe) * (uint32_t)sizeof(T);
              if (fl & 4) {  // my left edge is the left neighbour's right halo
                st_cluster(left_base + so + (uint32_t)(XW * (int)sizeof(T)), r0);
                if (row1) st_cluster(left_base + so + (uint32_t)((XT + XW) * (int)sizeof(T)), r1);
              }
              if (fl & 8) {  // my right edge is the right neighbour's left halo
                st_cluster(right_base + so - (uint32_t)(XW * (int)sizeof(T)), r0);
                if (row1) st_cluster(right_base + so + (uint32_t)((XT - XW) * (int)sizeof(T)), r1);
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
    cp_async_wait_group<PD - 1>();
    if (C > 1) cluster_arrive_release();
    else __syncthreads();  // a single block needs no second barrier: see the loop comment
    if (xw > 0) {
      if (w > 0) {  // planes the top level finished in step w-1
        for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) {
          if (wz < 0 || wz >= nz) continue;
          const int64_t gz = (int64_t)(wz + R) * gplane;
          for (int yy = warp; yy < YW; yy += nwarps) {
            const int m = row_mask[yy];
            if (m == 0) continue;
            const int64_t go = gz + (int64_t)(Y0 + yy + R) * ldx + (x0 + R);
            const T* src = sm + wsl * pe + yy * XT + R;
            for (int xl = lane; xl < xw; xl += 32) {
              if (m & 1) go0[go + xl] = src[xl];
              if (m & 2) go1[go + xl] = src[be + xl];
            }
          }
        }
      }
      for (int f = 0; f < nf; ++f, ++lz, lsl = (lsl + 1 == NZ) ? 0 : lsl + 1) {  // planes of step w+PD
        if (lz >= nz + R) continue;
        const int64_t gz = (int64_t)(lz + R) * gplane;
        for (int rr = warp; rr < 2 * nrow; rr += nwarps) {
          const int p = rr >= nrow;
          const int y = ylo + rr - p * nrow;
          const T* src = (p ? gb1 : gb0) + gz + (int64_t)(y + R) * ldx + x0;
          T* dst = sm + p * be + lsl * pe + (y - Y0) * XT;
          for (int xx = lane; xx < ncol; xx += 32) cp_async(dst + xx, src + xx);
        }
      }
    }
    cp_async_commit();
    if (C > 1) cluster_wait_acquire();
  }
  cp_async_wait_group<0>();
  if (xw > 0) {  // planes the top level finished in the last step
    for (int f = 0; f < nf; ++f, ++wz, wsl = (wsl + 1 == NZ) ? 0 : wsl + 1) {
      if (wz < 0 || wz >= nz) continue;
      const int64_t gz = (int64_t)(wz + R) * gplane;
      for (int yy = warp; yy < YW; yy += nwarps) {
        const int m = row_mask[yy];
        if (m == 0) continue;
        const int64_t go = gz + (int64_t)(Y0 + yy + R) * ldx + (x0 + R);
        const T* src = sm + wsl * pe + yy * XT + R;
        for (int xl = lane; xl < xw; xl += 32) {
          if (m & 1) go0[go + xl] = src[xl];
          if (m & 2) go1[go + xl] = src[be + xl];
        }
      }
    }
  }
}

MwdShape mwd_shape(int stencil, int dtype, int dw, int nf, int XW) {
  const int R = radius_of(stencil);
  const int H = dw / R;
  const int K = R + nf;
  MwdShape s;
  s.NZ = (MWD_PREFETCH + 1) * nf + R + (R > nf ? R : nf) + (H - 2) * K;
  s.YW = dw + 2 * R;
  s.XT = XW + 2 * R;
  const int elem = dtype == GIRIH_F64 ? 8 : 4;
  s.smem_bytes = 2LL * s.NZ * s.YW * s.XT * elem + (3LL * H + 1 + s.YW) * 4;
  return s;
}

// Row pairs of the widest (unclipped) diamond: levels k = 1..H-1 have 2R*min(k, H-k) rows.
int mwd_max_pairs(int R, int dw) {
  const int H = dw / R;
  int n = 0;
  for (int k = 1; k < H; ++k) n += R * (k < H - k ? k : H - k);
  return n;
}

// Pairs per thread for a configuration (1, 2 or 4), or 0 if the tile needs more.
int mwd_pairs_per_thread(int R, int dw, int XW, int threads) {
  const int64_t ng = (int64_t)mwd_max_pairs(R, dw) * XW;
  for (int G : {1, 2, 4})
    if (threads <= 1024 / G && ng <= (int64_t)G * threads) return G;
  return 0;
}

template <int S, typename T, int G>
static void* kernel_ptr_g() {
  return reinterpret_cast<void*>(&mwd_fed_kernel<S, T, G>);
}
template <int S, typename T>
static void* kernel_ptr(int G) {
  return G == 1 ? kernel_ptr_g<S, T, 1>() : (G == 2 ? kernel_ptr_g<S, T, 2>() : kernel_ptr_g<S, T, 4>());
}

static void* pick(int stencil, int dtype, int G) {
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case 0: return f64 ? kernel_ptr<0, double>(G) : kernel_ptr<0, float>(G);
    case 1: return f64 ? kernel_ptr<1, double>(G) : kernel_ptr<1, float>(G);
    case 2: return f64 ? kernel_ptr<2, double>(G) : kernel_ptr<2, float>(G);
    default: return f64 ? kernel_ptr<3, double>(G) : kernel_ptr<3, float>(G);
  }
}

static cudaLaunchConfig_t launch_config(int C, int threads, int64_t smem, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t mwd_prepare(int stencil, int dtype, int C, int threads, int G, int64_t smem, int* max_clusters) {
  const void* k = pick(stencil, dtype, G);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  if (max_clusters) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config(C, threads, smem, attr);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    if (e != cudaSuccess) return e;
    *max_clusters = n;
  }
  return cudaSuccess;
}

cudaError_t launch_mwd_row(int stencil, int dtype, const MwdArgs& a, int ndiam, int threads, int G, cudaStream_t st) {
  const MwdShape sh = mwd_shape(stencil, dtype, a.dw, a.nf, a.XW);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_config(a.C, threads, sh.smem_bytes, attr);
  cfg.gridDim = dim3((unsigned)(ndiam * a.C), 1, 1);
  cfg.stream = st;
  const void* k = pick(stencil, dtype, G);
  void* args[] = {const_cast<MwdArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace girih
