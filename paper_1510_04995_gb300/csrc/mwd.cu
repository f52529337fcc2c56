// Host side of the wavefront-diamond sweep: tile shapes, kernel selection, cluster launches.
// The kernel itself is in mwd_kernel.cuh (instantiated in mwd_r1.cu and mwd_r4.cu).
#include <algorithm>

#include "internal.h"

namespace girih {

void* mwd_kernel_r1(int stencil, int dtype, int G);
void* mwd_kernel_r4(int stencil, int dtype, int G);
void* mwd_vec_kernel_r1(int stencil, int dtype, int G, bool tma);
void* mwd_vec_kernel_r4(int stencil, int dtype, int G, bool tma);
void* mwd_kernel_cg(int dtype, int G);
void* mwd_vec_kernel_cg(int dtype, int G, bool tma);
void* mwd_vec_kernel_box(int dtype, int G, bool tma);
void* mwd_vec_kernel_rb(int dtype, int G, bool tma);

void* mwd_async_kernel_ptr(int stencil, int dtype, int G);
void* mwd_ovl_kernel_ptr(int stencil, int dtype, int G, bool zseg);

static void* pick(int stencil, int dtype, int G, int mv) {
  if (mv == MV_ASYNC) return mwd_async_kernel_ptr(stencil, dtype, G);
  if (mv_ovl(mv)) return mwd_ovl_kernel_ptr(stencil, dtype, G, mv == MV_OVLZ);
  if (mv_shifted(mv)) {
    const bool tma = mv == MV_BULK;
    if (stencil == GIRIH_25PT_CGRID) return mwd_vec_kernel_cg(dtype, G, tma);
    if (stencil == GIRIH_27PT_BOX) return mwd_vec_kernel_box(dtype, G, tma);
    if (stencil == GIRIH_7PT_RBGS) return mwd_vec_kernel_rb(dtype, G, tma);
    return stencil < 2 ? mwd_vec_kernel_r1(stencil, dtype, G, tma) : mwd_vec_kernel_r4(stencil, dtype, G, tma);
  }
  if (stencil == GIRIH_25PT_CGRID) return mwd_kernel_cg(dtype, G);
  return stencil < 2 ? mwd_kernel_r1(stencil, dtype, G) : mwd_kernel_r4(stencil, dtype, G);
}

MwdShape mwd_shape(int stencil, int dtype, int dw, int nf, int XW, int mv, int lead) {
  const int R = radius_of(stencil);
  const int H = dw / R;
  const int K = R + nf;
  const int elem = dtype == GIRIH_F64 ? 8 : 4;
  const int a16 = 16 / elem;
  MwdShape s;
  if (mv_ovl(mv)) {
    // the MV_ASYNC ring on widened slabs; load mbarriers, progress words (2) and item slot,
    // level tables (5H+3)
    const int L = lead;
    s.HM = ovl_margin(H, R, a16);
    s.NZ = L + 2 * R + 1 + (H - 2) * K;
    s.YW = dw + 2 * R;
    s.XT = XW + 2 * s.HM;
    const int per128 = 128 / elem;
    s.PE = (s.YW * s.XT + per128 - 1) / per128 * per128;
    const int64_t ring = 2LL * s.NZ * s.PE * elem;
    s.smem_bytes = (ring + 15) / 16 * 16 + 8LL * kAsyncLoadBars + 16 + (5LL * H + 3) * 4;
    return s;
  }
  if (mv == MV_ASYNC) {
    // ring (one plane per level and step): a slot is restaged, L steps ahead and while the
    // computing warps run the current step, once its plane is below every level's read window and
    // has been written back in an earlier step (mwd_async.cuh); halo mbarriers (2), level tables
    // (3H+1), row masks (YW), item slot (1)
    const int L = lead;
    s.NZ = L + 2 * R + 1 + (H - 2) * K;
    s.YW = dw + 2 * R;
    s.XT = XW + 2 * ((R + a16 - 1) / a16 * a16);
    const int per128 = 128 / elem;  // slots start on 128-byte boundaries (tensor copy destinations)
    s.PE = (s.YW * s.XT + per128 - 1) / per128 * per128;
    const int64_t ring = 2LL * s.NZ * s.PE * elem;
    s.smem_bytes = (ring + 15) / 16 * 16 + 8LL * (2 + kAsyncLoadBars) + (3LL * H + 2) * 4;
    return s;
  }
  const bool bulk = mv == MV_BULK;
  const int pd = bulk ? MWD_PREFETCH_BULK : MWD_PREFETCH;
  s.NZ = (pd + 1) * nf + R + (R > nf ? R : nf) + (H - 2) * K + (bulk ? MWD_BULK_SLACK : MWD_PLAIN_SLACK) * nf;
  s.YW = dw + 2 * R;
  // shared row: [halo | slab | halo], rows starting on 16-byte boundaries.  Element path: the
  // slab starts on a 16-byte boundary when groups are vectors.  Vector path: HM = R rounded up
  // to 16 bytes columns each side, so global and shared rows share their 16-byte alignment.
  if (mv_shifted(mv)) {
    const int hm = (R + a16 - 1) / a16 * a16;
    s.XT = XW + 2 * hm;
  } else {
    const int off = mwd_vx(stencil, dtype, mv) == 1 ? R : a16;
    s.XT = (off + XW + R + a16 - 1) / a16 * a16;
  }
  const int64_t ring = 2LL * s.NZ * s.YW * s.XT * elem;
  // ring, one mbarrier per plane, level tables (3H+1), row masks (YW), RELAXED progress
  // counters (2), persistent-schedule item slot (1)
  s.smem_bytes = (ring + 15) / 16 * 16 + 8LL * s.NZ + (3LL * H + 1 + s.YW + 3) * 4;
  return s;
}

int mwd_async_lead(int stencil, int dtype, int dw, int nf, int XW, int threads, int G, int64_t smem_optin,
                   int mv) {
  const void* k = pick(stencil, dtype, G, mv);
  auto per_sm = [&](int L) {
    const MwdShape sh = mwd_shape(stencil, dtype, dw, nf, XW, mv, L);
    if (sh.smem_bytes > smem_optin) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem_bytes) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, (size_t)sh.smem_bytes) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  };
  const int base = per_sm(kAsyncLeadMin);
  if (base < 1) return kAsyncLeadMin;
  for (int L = kAsyncLeadMax; L > kAsyncLeadMin; --L)
    if (per_sm(L) >= base) return L;
  return kAsyncLeadMin;
}

int64_t mwd_ovl_tasks(int R, int dw, int XW, int vx, int a16) {
  const int H = dw / R, hm = ovl_margin(H, R, a16), smax = H - 2;
  int64_t n = 0;
  for (int k = 1; k < H; ++k) {  // level s = k - 1
    const int e = (smax - (k - 1)) * R;
    const int nv = (hm + XW + e + vx - 1) / vx - (hm - e) / vx;
    n += (int64_t)R * (k < H - k ? k : H - k) * nv;
  }
  return n;
}

// Row pairs of the widest (unclipped) diamond: levels k = 1..H-1 have 2R*min(k, H-k) rows.
int mwd_max_pairs(int R, int dw) {
  const int H = dw / R;
  int n = 0;
  for (int k = 1; k < H; ++k) n += R * (k < H - k ? k : H - k);
  return n;
}

// Groups (row pair x VX columns) per computing thread (1, 2, 4 or 8) for a block of `threads`
// or 0 if the tile needs more.
int mwd_pairs_per_thread(int stencil, int dtype, int dw, int XW, int threads, int mv) {
  const int R = radius_of(stencil);
  const int vx = mwd_vx(stencil, dtype, mv), lbf = mwd_lbf(stencil, dtype, mv);
  const int64_t ng = (int64_t)mwd_max_pairs(R, dw) * (XW / vx);
  if (mv_ovl(mv)) {  // the block's last two warps move data; the others compute
    const int64_t nt = mwd_ovl_tasks(R, dw, XW, vx, 16 / (dtype == GIRIH_F64 ? 8 : 4));
    for (int G : {1, 2, 4})
      if (threads <= async_max_threads(G, ncoef_of(stencil) > 0, R == 4) && nt <= (int64_t)G * (threads - kOvlMovers))
        return G;
    return 0;
  }
  if (mv == MV_ASYNC) {  // the block's last two warps move data; the others compute
    for (int G : {1, 2, 4})
      if (threads <= async_max_threads(G, ncoef_of(stencil) > 0) && ng <= (int64_t)G * (threads - kAsyncMovers)) return G;
    return 0;
  }
  const int ct = threads;
  for (int G : {1, 2, 4, 8}) {
    if (G == 8 && R == 4) break;  // radius-4 kernels are built for at most 4 groups per thread
    if (G > 2 && R == 4 && vx > 1 && mv == MV_ELEM) break;  // radius-4 vector windows: 2 per thread
    if (threads <= mwd_max_threads(G, lbf) && ng <= (int64_t)G * ct) return G;
  }
  return 0;
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

cudaError_t mwd_prepare(int stencil, int dtype, int C, int threads, int G, int mv, int64_t smem,
                        int* max_clusters) {
  const void* k = pick(stencil, dtype, G, mv);
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

cudaError_t launch_mwd_row(int stencil, int dtype, const MwdArgs& a, int ndiam, int threads, int G, int mv,
                           int64_t smem, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_config(a.C, threads, smem, attr);
  cfg.gridDim = dim3((unsigned)(ndiam * a.C), 1, 1);
  cfg.stream = st;
  void* args[] = {const_cast<MwdArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, pick(stencil, dtype, G, mv), args);
}

}  // namespace girih
