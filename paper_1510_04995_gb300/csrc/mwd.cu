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

template <int S, typename T>
struct MwdAcc {
  const T* V;        // level t buffer of the ring
  const T* U;        // level t-1 buffer of the ring (second order)
  const T* coef;
  int64_t gs, p;     // coefficient grid stride, padded global index of the point
  int pe, xt, NZ;    // plane elems, row pitch, ring depth
  int sl, off;       // ring slot of the point's plane, offset of the point within a plane
  __device__ __forceinline__ int slot(int d) const {
    int s = sl + d;
    s = (s < 0) ? s + NZ : s;
    return (s >= NZ) ? s - NZ : s;
  }
  __device__ __forceinline__ T c() const { return V[sl * pe + off]; }
  __device__ __forceinline__ T x(int d) const { return V[sl * pe + off + d]; }
  __device__ __forceinline__ T y(int d) const { return V[sl * pe + off + d * xt]; }
  __device__ __forceinline__ T z(int d) const { return V[slot(d) * pe + off]; }
  __device__ __forceinline__ T u() const { return U[sl * pe + off]; }
  __device__ __forceinline__ T k(int g) const { return __ldg(coef + g * gs + p); }
};

__device__ __forceinline__ int lev_lo_of(int a, int b, int dw, int R, int t) {
  return max(a * dw - R * t, b * dw + R * t);
}
__device__ __forceinline__ int lev_hi_of(int a, int b, int dw, int R, int t) {
  return min((a + 1) * dw - R * t, (b + 1) * dw + R * t);
}

template <int S, typename T>
__global__ void __launch_bounds__(512) mwd_fed_kernel(const MwdArgs A) {
  constexpr int R = Traits<S>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int NZ = A.NZ, YW = A.YW, XT = A.XT, XW = A.XW, C = A.C, nf = A.nf, K = A.K;
  const int pe = YW * XT;
  const int be = NZ * pe;
  int* lev_lo = reinterpret_cast<int*>(sm + 2 * be);
  int* lev_w = lev_lo + A.H;
  int* row_mask = lev_w + A.H;

  const int nx = (int)A.g.nx, ny = (int)A.g.ny, nz = (int)A.g.nz;
  const int64_t ldx = A.g.ldx, sy = A.g.sy, gplane = sy * ldx;
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

  for (int s = tid; s < nlev; s += NT) {
    const int t = tb + s;
    const int lo = max(lev_lo_of(a, b, dw, R, t), 0);
    const int hi = min(lev_hi_of(a, b, dw, R, t), ny);
    lev_lo[s] = lo;
    lev_w[s] = max(hi - lo, 0);
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

  const T* gbuf[2] = {static_cast<const T*>(A.buf0), static_cast<const T*>(A.buf1)};
  T* gout[2] = {static_cast<T*>(A.buf0), static_cast<T*>(A.buf1)};
  const T* coef = static_cast<const T*>(A.coef);
  T cst[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) cst[i] = static_cast<T>(A.c[i]);

  // Rows and columns of the padded grid this block stages: y in [Y0, Y0+YW) clipped to the
  // padded grid, x in [x0-R, x0+xw+R) (slab plus x halo).
  const int ylo = max(Y0, -R), yhi = min(Y0 + YW, ny + R);
  const int nrow = max(yhi - ylo, 0);
  const int ncol = (xw > 0) ? xw + 2 * R : 0;

  auto load_plane = [&](int z) {
    if (z < -R || z >= nz + R || ncol == 0) return;
    const int slot = (z + R) % NZ;
    const int per = nrow * ncol;
    for (int i = tid; i < 2 * per; i += NT) {
      const int p = i / per, rem = i - p * per;
      const int r = rem / ncol, xx = rem - r * ncol;
      const int y = ylo + r;
      const int64_t gi = (int64_t)(z + R) * gplane + (int64_t)(y + R) * ldx + (x0 + xx);
      cp_async(sm + p * be + slot * pe + (y - Y0) * XT + xx, gbuf[p] + gi);
    }
  };
  auto write_plane = [&](int z) {
    if (z < 0 || z >= nz || xw <= 0) return;
    const int slot = (z + R) % NZ;
    const int per = YW * xw;
    for (int i = tid; i < per; i += NT) {
      const int yy = i / xw, xl = i - yy * xw;
      const int m = row_mask[yy];
      if (m == 0) continue;
      const int64_t gi = (int64_t)(z + R) * gplane + (int64_t)(Y0 + yy + R) * ldx + (x0 + xl + R);
      const int so = slot * pe + yy * XT + xl + R;
      if (m & 1) gout[0][gi] = sm[so];
      if (m & 2) gout[1][gi] = sm[be + so];
    }
  };
  auto sync_all = [&]() {
    if (C > 1) cluster_barrier();
    else __syncthreads();
  };

  __syncthreads();  // level tables ready
  for (int z = -R; z < nf + R; ++z) load_plane(z);
  cp_async_wait_all();
  sync_all();

  const uint32_t sm_base = smem_addr(sm);
  const uint32_t left_base = (C > 1 && rank > 0) ? map_to_rank(sm_base, rank - 1) : 0u;
  const uint32_t right_base = (C > 1 && rank < C - 1) ? map_to_rank(sm_base, rank + 1) : 0u;

  const int W = (nz + smax * K + nf - 1) / nf;
  for (int w = 0; w < W; ++w) {
    if (xw > 0) {
      for (int f = 0; f < nf; ++f) load_plane((w + 1) * nf + R + f);
      if (w > 0)
        for (int f = 0; f < nf; ++f) write_plane((w - 1) * nf - smax * K + f);
      // compute: all active levels of this step, items linearised over (level, row, plane, x)
      int base = 0, it = tid;
      for (int s = 0; s < nlev; ++s) {
        const int zb = w * nf - s * K;
        if (zb + nf <= 0 || zb >= nz) continue;
        const int n = lev_w[s] * nf * XW;
        const int t = tb + s;
        const int pin = t & 1, pout = pin ^ 1;
        const int ylo_s = lev_lo[s];
        for (; it < base + n; it += NT) {
          const int i = it - base;
          const int xl = i % XW, r2 = i / XW;
          const int f = r2 % nf, row = r2 / nf;
          const int z = zb + f;
          if (xl >= xw || z < 0 || z >= nz) continue;
          const int y = ylo_s + row;
          const int sl = (z + R) % NZ;
          const int off = (y - Y0) * XT + xl + R;
          const int64_t gp = (int64_t)(z + R) * gplane + (int64_t)(y + R) * ldx + (x0 + xl + R);
          MwdAcc<S, T> acc{sm + pin * be, sm + pout * be, coef, A.g.gstride, gp, pe, XT, NZ, sl, off};
          const T res = point_update<S, T>(acc, cst);
          const int so = pout * be + sl * pe + off;
          sm[so] = res;
          if (C > 1) {
            if (xl < R && rank > 0)  // my left edge is the left neighbour's right halo
              st_cluster(left_base + (uint32_t)((so + XW) * (int)sizeof(T)), res);
            if (xl >= XW - R && rank < C - 1)  // my right edge is the right neighbour's left halo
              st_cluster(right_base + (uint32_t)((so - XW) * (int)sizeof(T)), res);
          }
        }
        base += n;
      }
    }
    cp_async_wait_all();
    sync_all();
  }
  if (xw > 0)
    for (int f = 0; f < nf; ++f) write_plane((W - 1) * nf - smax * K + f);
}

MwdShape mwd_shape(int stencil, int dtype, int dw, int nf, int XW) {
  const int R = radius_of(stencil);
  const int H = dw / R;
  const int K = R + nf;
  MwdShape s;
  s.NZ = 2 * nf + R + (R > nf ? R : nf) + (H - 2) * K;
  s.YW = dw + 2 * R;
  s.XT = XW + 2 * R;
  const int elem = dtype == GIRIH_F64 ? 8 : 4;
  s.smem_bytes = 2LL * s.NZ * s.YW * s.XT * elem + (2LL * H + s.YW) * 4;
  return s;
}

template <int S, typename T>
static void* kernel_ptr() {
  return reinterpret_cast<void*>(&mwd_fed_kernel<S, T>);
}

static void* pick(int stencil, int dtype) {
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case 0: return f64 ? kernel_ptr<0, double>() : kernel_ptr<0, float>();
    case 1: return f64 ? kernel_ptr<1, double>() : kernel_ptr<1, float>();
    case 2: return f64 ? kernel_ptr<2, double>() : kernel_ptr<2, float>();
    default: return f64 ? kernel_ptr<3, double>() : kernel_ptr<3, float>();
  }
}

cudaError_t mwd_prepare(int stencil, int dtype, int C, int threads, int64_t smem, int* max_clusters) {
  const void* k = pick(stencil, dtype);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  if (max_clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    if (e != cudaSuccess) return e;
    *max_clusters = n;
  }
  return cudaSuccess;
}

cudaError_t launch_mwd_row(int stencil, int dtype, const MwdArgs& a, int ndiam, int threads, cudaStream_t st) {
  const MwdShape sh = mwd_shape(stencil, dtype, a.dw, a.nf, a.XW);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ndiam * a.C), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)sh.smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool f64 = dtype == GIRIH_F64;
  switch (stencil) {
    case 0: return f64 ? cudaLaunchKernelEx(&cfg, mwd_fed_kernel<0, double>, a) : cudaLaunchKernelEx(&cfg, mwd_fed_kernel<0, float>, a);
    case 1: return f64 ? cudaLaunchKernelEx(&cfg, mwd_fed_kernel<1, double>, a) : cudaLaunchKernelEx(&cfg, mwd_fed_kernel<1, float>, a);
    case 2: return f64 ? cudaLaunchKernelEx(&cfg, mwd_fed_kernel<2, double>, a) : cudaLaunchKernelEx(&cfg, mwd_fed_kernel<2, float>, a);
    default: return f64 ? cudaLaunchKernelEx(&cfg, mwd_fed_kernel<3, double>, a) : cudaLaunchKernelEx(&cfg, mwd_fed_kernel<3, float>, a);
  }
}

}  // namespace girih
