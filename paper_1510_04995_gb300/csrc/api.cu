// C ABI of the stencil sweep library: plans, validation, the per-row launch loop of the
// wavefront-diamond sweep, the naive loop, and the paper's cache-block / code-balance models.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "internal.h"
#include "plan.h"

namespace girih {

thread_local std::string g_err;

void g_err_clear() { g_err.clear(); }

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(GIRIH_ECUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

static int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Diamond rows of the sweep: rows 0..rho_max have at least one step in [0, T).
int64_t mwd_rows(int64_t T, int dw, int R) {
  if (T <= 0) return 0;
  const int64_t Hh = dw / R / 2;
  int64_t rho = 0;
  while ((rho + 1 - 1) * Hh + 1 <= T - 1) ++rho;  // next row's first step still below T
  return rho + 1;
}

// Diamonds of row rho whose y projection [a*dw - rho*dw/2, +dw) meets [0, ny).
void mwd_row_span(int64_t rho, int dw, int64_t ny, int64_t* a_min, int64_t* ndiam) {
  const int64_t h = rho * (dw / 2);
  const int64_t lo = floor_div(h, dw);
  const int64_t hi = floor_div(ny + h + dw - 1, dw) - 1;  // ceil((ny + h)/dw) - 1
  *a_min = lo;
  *ndiam = std::max<int64_t>(hi - lo + 1, 0);
}

// x slab per block (blocks past the end of the grid stay idle but take part in the cluster's
// synchronisation).  Element path: nx split evenly, rounded up to 16 elements.  Vector and
// bulk-copy paths: the slabs partition the padded columns [R, nx + R) at 16-byte boundaries
// (block r owns padded [r*XW, (r+1)*XW)), so nx + R columns are split, rounded up to 16 bytes.
int slab_width(const Plan* p, int C, int mv) {
  if (mv_shifted(mv)) {
    const int a16 = 16 / p->elem;
    const int64_t w = (p->nx + p->R + C - 1) / C;
    return (int)((w + a16 - 1) / a16 * a16);
  }
  const int64_t w = (p->nx + C - 1) / C;
  return (int)((w + 15) / 16 * 16);
}

// Data path of a configuration: FED_BULK moves rows with the bulk-copy engine; FED and RELAXED
// use 16-byte vectors when rows are 16-byte multiples (and, at run time, the buffers 16-byte
// aligned), else per-element staging.
static int mwd_path(const Plan* p, const girih_config* c, bool ptrs16) {
  if (c->variant == GIRIH_FED_BULK) return MV_BULK;
  if (c->variant == GIRIH_FED_ELEM || c->variant == GIRIH_RELAXED_ELEM) return MV_ELEM;
  const int64_t plane = (p->ny + 2 * p->R) * p->ldx;
  const bool vec = p->bulk_layout && ptrs16 && plane < (1LL << 30);
  if (c->variant == GIRIH_RELAXED_PERSISTENT) return vec ? MV_ASYNC : MV_ELEM;
  // segments of nz planes or more leave one segment per tile: the whole-tile kernel (the
  // segmented one reads the items' segment list, which is uploaded only for two or more)
  if (c->variant == GIRIH_OVERLAP_PERSISTENT)
    return vec ? ((c->zseg > 0 && c->zseg < p->nz) ? MV_OVLZ : MV_OVL) : MV_ELEM;
  return vec ? MV_VEC : MV_ELEM;
}

static bool persistent_variant(int v) {
  return v == GIRIH_FED_PERSISTENT || v == GIRIH_RELAXED_PERSISTENT || v == GIRIH_OVERLAP_PERSISTENT;
}
// variants of the warp-specialised kernels (radius-1 first-order stencils, tensor-map staging)
static bool tma_variant(int v) { return v == GIRIH_RELAXED_PERSISTENT || v == GIRIH_OVERLAP_PERSISTENT; }
static const char* variant_name(int v) {
  return v == GIRIH_OVERLAP_PERSISTENT ? "OVERLAP_PERSISTENT" : "RELAXED_PERSISTENT";
}

int check_config(const Plan* p, const girih_config* c, int64_t* smem_out, int* xw_out, int* g_out, int* mv_out,
                 bool ptrs16, int* lead_out) {
  if (!c) return fail(GIRIH_EINVAL, "config is NULL");
  if (c->algo == GIRIH_ALGO_NAIVE) {
    if (smem_out) *smem_out = 0;
    return GIRIH_OK;
  }
  if (c->algo != GIRIH_ALGO_MWD) return fail(GIRIH_EINVAL, "unknown algo %d", c->algo);
  if (c->variant < GIRIH_FED || c->variant > GIRIH_OVERLAP_PERSISTENT)
    return fail(GIRIH_EINVAL, "unknown variant %d", c->variant);
  if (c->zseg < 0) return fail(GIRIH_EINVAL, "zseg=%d must be >= 0", c->zseg);
  if (c->zseg > 0 && c->variant != GIRIH_OVERLAP_PERSISTENT)
    return fail(GIRIH_EINVAL, "zseg=%d: only OVERLAP_PERSISTENT splits tiles along z", c->zseg);
  if (c->variant == GIRIH_FED_PERSISTENT && mwd_path(p, c, ptrs16) != MV_VEC)
    return fail(GIRIH_EINVAL, "FED_PERSISTENT needs rows of 16-byte multiples and 16-byte aligned buffers");
  if (tma_variant(c->variant)) {
    const char* vn = variant_name(c->variant);
    if (c->variant == GIRIH_RELAXED_PERSISTENT && !async_stencil(p->stencil))
      return fail(GIRIH_EINVAL, "%s is built for the radius-1 first-order stencils (7-point constant, 7-point "
                  "variable, red-black Gauss-Seidel)", vn);
    if (c->variant == GIRIH_OVERLAP_PERSISTENT && !ovl_stencil(p->stencil))
      return fail(GIRIH_EINVAL, "%s is built for the 7-point, red-black and 25-point stencils (not the box "
                  "stencil)", vn);
    if (!mv_tma(mwd_path(p, c, ptrs16)))
      return fail(GIRIH_EINVAL, "%s needs rows of 16-byte multiples and 16-byte aligned buffers", vn);
    if (c->nf != 1) return fail(GIRIH_EINVAL, "%s advances one plane per level and step (nf = 1)", vn);
    const int movers = c->variant == GIRIH_OVERLAP_PERSISTENT ? kOvlMovers : kAsyncMovers;
    if (c->threads <= movers)
      return fail(GIRIH_EINVAL, "%s needs more than %d threads (%d warp(s) move data)", vn, movers, movers / 32);
  }
  if (vec_only(p->stencil) && mwd_path(p, c, ptrs16) == MV_ELEM)
    return fail(GIRIH_EINVAL, "the blocked sweep of the box and red-black stencils needs the vector path: rows of "
                "16-byte multiples, 16-byte aligned buffers and a variant other than FED_ELEM / RELAXED_ELEM");
  const bool bulk = c->variant == GIRIH_FED_BULK;
  if (bulk && !p->bulk_layout)
    return fail(GIRIH_EINVAL, "FED_BULK needs ldx*elem to be a multiple of 16 bytes (ldx=%lld)", (long long)p->ldx);
  if (bulk && (p->ny + 2 * p->R) * p->ldx >= (1LL << 30))
    return fail(GIRIH_EINVAL, "FED_BULK needs planes of fewer than 2^30 elements");
  const int R = p->R;
  if (c->dw < 2 * R || c->dw % (2 * R) != 0)
    return fail(GIRIH_EINVAL, "dw=%d must be a positive multiple of 2R=%d", c->dw, 2 * R);
  if (c->nf < 1 || c->nf > 4) return fail(GIRIH_EINVAL, "nf=%d outside 1..4", c->nf);
  if (!(c->cluster == 1 || c->cluster == 2 || c->cluster == 4 || c->cluster == 8 || c->cluster == 16))
    return fail(GIRIH_EINVAL, "cluster=%d not in {1,2,4,8,16}", c->cluster);
  if (c->threads < 64 || c->threads > 1024 || c->threads % 32 != 0)
    return fail(GIRIH_EINVAL, "threads=%d must be a multiple of 32 in 64..1024", c->threads);
  const int mv = mwd_path(p, c, ptrs16);
  const int XW = slab_width(p, c->cluster, mv);
  const int cthreads = c->threads;
  const int G = mwd_pairs_per_thread(p->stencil, p->dtype, c->dw, XW, c->threads, mv);
  if (G == 0 && mv_ovl(mv))
    return fail(GIRIH_EINVAL, "dw=%d with a %d-wide slab has %lld tasks on its widened levels: more than the %d "
                "computing threads of a %d-thread block hold at 1, 2 or 4 per thread (blocks of at most %d, %d, %d "
                "threads)", c->dw, XW, (long long)mwd_ovl_tasks(R, c->dw, XW, mwd_vx(p->stencil, p->dtype, mv), 16 / p->elem),
                c->threads - kOvlMovers, c->threads, async_max_threads(1, ncoef_of(p->stencil) > 0, R == 4),
                async_max_threads(2, ncoef_of(p->stencil) > 0, R == 4),
                async_max_threads(4, ncoef_of(p->stencil) > 0, R == 4));
  if (G == 0 && mv == MV_ASYNC)
    return fail(GIRIH_EINVAL, "dw=%d with a %d-wide slab has %d row pairs x %d vectors: more tasks than the %d "
                "computing threads of a %d-thread block hold (blocks of at most %d, %d, %d threads for 1, 2, 4 tasks "
                "per thread)", c->dw, XW, mwd_max_pairs(R, c->dw), XW / mwd_vx(p->stencil, p->dtype, mv),
                c->threads - kAsyncMovers, c->threads, async_max_threads(1, ncoef_of(p->stencil) > 0), async_max_threads(2, ncoef_of(p->stencil) > 0),
                async_max_threads(4, ncoef_of(p->stencil) > 0));
  if (G == 0)
    return fail(GIRIH_EINVAL, "dw=%d with a %d-wide slab has %d row pairs x %d column groups: no groups-per-thread "
                "count fits %d threads within the kernel's launch bound (%d threads for one group per thread)",
                c->dw, XW, mwd_max_pairs(R, c->dw), XW / mwd_vx(p->stencil, p->dtype, mv), cthreads,
                mwd_max_threads(1, mwd_lbf(p->stencil, p->dtype, mv)));
  if (R == 4 && G > 4) return fail(GIRIH_EINVAL, "25-point tiles allow at most 4 row pairs per thread (registers)");
  if (p->dtype == GIRIH_F64 && R == 4 && G > 2)
    return fail(GIRIH_EINVAL, "25-point FP64 tiles allow at most 2 row pairs per thread (registers)");
  if (p->ny > (1 << 28) || p->nx > (1 << 28) || p->nz > (1 << 28))
    return fail(GIRIH_EINVAL, "grid too large for the blocked kernel");
  const int lead = mv_tma(mv) ? mwd_async_lead(p->stencil, p->dtype, c->dw, c->nf, XW, c->threads, G, p->smem_optin, mv)
                               : kAsyncLeadMin;
  const MwdShape sh = mwd_shape(p->stencil, p->dtype, c->dw, c->nf, XW, mv, lead);
  if (mv_tma(mv) && sh.XT > 256)
    return fail(GIRIH_EINVAL, "%s stages a slab of %d columns with its halo per tensor copy (at "
                "most 256): use a larger cluster", variant_name(c->variant), sh.XT);
  if (sh.smem_bytes > p->smem_optin)
    return fail(GIRIH_EINVAL, "config needs %lld bytes of shared memory per block (device limit %lld)",
                (long long)sh.smem_bytes, (long long)p->smem_optin);
  int maxc = 0;
  cudaError_t e = mwd_prepare(p->stencil, p->dtype, c->cluster, c->threads, G, mv, sh.smem_bytes, &maxc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GIRIH_EINVAL, "cluster of %d blocks with %lld bytes cannot be configured: %s", c->cluster,
                (long long)sh.smem_bytes, cudaGetErrorString(e));
  }
  if (maxc < 1) return fail(GIRIH_EINVAL, "cluster of %d blocks cannot be scheduled", c->cluster);
  if (smem_out) *smem_out = sh.smem_bytes;
  if (xw_out) *xw_out = XW;
  if (g_out) *g_out = G;
  if (mv_out) *mv_out = mv;
  if (lead_out) *lead_out = lead;
  return GIRIH_OK;
}

// Default configuration: the widest diamond whose tile fits (Sect. 4.2.2 prunes with the
// cache-block model; here the block's shared memory is the cache), smallest cluster first.
static girih_config default_config(Plan* p) {
  girih_config best{GIRIH_ALGO_NAIVE, 0, 1, 1, 256, GIRIH_FED};
  int best_dw = 0;
  const int R = p->R;
  for (int th : {512, 256, 1024})
    for (int C : {1, 2, 4, 8, 16}) {
      for (int dw = 2 * R; dw <= 64 * R; dw += 2 * R) {
        girih_config c{GIRIH_ALGO_MWD, dw, 1, C, th, GIRIH_FED};
        int64_t smem = 0;
        if (check_config(p, &c, &smem, nullptr, nullptr) != GIRIH_OK) continue;
        if (dw > best_dw && dw <= (R == 1 ? 16 : 32)) {
          best_dw = dw;
          best = c;
        }
      }
    }
  g_err.clear();
  return best;
}

static int launch_persistent(Plan* p, MwdArgs a, int64_t rows, const girih_config& cfg, int G, int mv,
                             int64_t smem, cudaStream_t st, cudaError_t* e_out);

// 3D tensor maps of the two buffers for the RELAXED_PERSISTENT staging copies: the padded grid
// (ldx x (ny+2R) x (nz+2R)), a box of one slab with its halo (XT columns) x YW rows x 1 plane;
// elements outside the grid read as zeros.
// The driver's tensor-map encoder, looked up through the runtime (the library does not link the
// driver library, so that it loads on machines without a GPU driver).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  }
  return fn;
}

static int encode_plane_maps(const Plan* p, void* u, void* up, int XT, int YW, CUtensorMap* tm) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return fail(GIRIH_ECUDA, "the driver's cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {(cuuint64_t)p->ldx, (cuuint64_t)(p->ny + 2 * p->R), (cuuint64_t)(p->nz + 2 * p->R)};
  const cuuint64_t strides[2] = {(cuuint64_t)p->ldx * p->elem, (cuuint64_t)(p->ny + 2 * p->R) * p->ldx * p->elem};
  const cuuint32_t box[3] = {(cuuint32_t)XT, (cuuint32_t)YW, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt = p->dtype == GIRIH_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  void* bufs[2] = {u, up};
  for (int i = 0; i < 2; ++i) {
    const CUresult r = encode(&tm[i], dt, 3, bufs[i], dims, strides, box, estr,
                                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GIRIH_ECUDA, "tensor map of buffer %d: CUresult %d", i, (int)r);
  }
  return GIRIH_OK;
}

int run_sweep(Plan* p, int64_t T, void* u, void* u_prev, const void* coeffs, const double* c,
              const girih_config& cfg, cudaStream_t st) {
  Grid g{p->nx, p->ny, p->nz, p->ldx, p->ny + 2 * p->R, p->gstride};
  cudaError_t e = cudaSuccess;
  if (cfg.algo == GIRIH_ALGO_NAIVE) {
    NaiveArgs a{};
    a.g = g;
    a.coef = coeffs;
    for (int i = 0; i < 5; ++i) {
      a.c[i] = c[i];
      a.cf[i] = (float)c[i];
    }
    a.v16 = (p->bulk_layout &&
             ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev)) & 15) == 0) ? 1 : 0;
    a.zc = naive_z_chunk(p->nx, p->ny, p->nz, p->R, naive_tile_x(p->stencil, p->dtype, a.v16 != 0),
                         naive_tile_y(p->stencil, p->dtype),
                         naive_resident_blocks(p->stencil, p->dtype, a.v16 != 0), p->sm_count);
    void* buf[2] = {u, u_prev};
    for (int64_t t = 0; t < T && e == cudaSuccess; ++t) {
      a.V = buf[t % 2];
      a.U = buf[(t + 1) % 2];
      a.t = (int32_t)t;
      e = launch_naive_step(p->stencil, p->dtype, a, st);
    }
  } else {
    int64_t smem = 0;
    int XW = 0, G = 0, mv = 0, lead = 0;
    const bool ptrs16 = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev)) & 15) == 0;
    const int rc = check_config(p, &cfg, &smem, &XW, &G, &mv, ptrs16, &lead);
    if (rc != GIRIH_OK) return rc;
    e = mwd_prepare(p->stencil, p->dtype, cfg.cluster, cfg.threads, G, mv, smem, nullptr);
    const MwdShape sh = mwd_shape(p->stencil, p->dtype, cfg.dw, cfg.nf, XW, mv, lead);
    MwdArgs a{};
    a.g = g;
    a.buf0 = u;
    a.buf1 = u_prev;
    a.coef = coeffs;
    for (int i = 0; i < 5; ++i) {
      a.c[i] = c[i];
      a.cf[i] = (float)c[i];
    }
    a.T = (int32_t)T;
    a.dw = cfg.dw;
    a.nf = cfg.nf;
    a.K = p->R + cfg.nf;
    a.H = cfg.dw / p->R;
    a.C = cfg.cluster;
    a.XW = XW;
    a.NZ = sh.NZ;
    a.YW = sh.YW;
    a.XT = sh.XT;
    a.err = p->err;
    a.lead = lead;
    a.PE = sh.PE;
    a.HMO = sh.HM;
    if (mv_tma(mv)) {
      const int rc3 = encode_plane_maps(p, u, u_prev, sh.XT, sh.YW, a.tm);
      if (rc3 != GIRIH_OK) return rc3;
    }
    a.relaxed = (cfg.variant == GIRIH_RELAXED || cfg.variant == GIRIH_RELAXED_ELEM) ? 1 : 0;
    const int64_t rows = mwd_rows(T, cfg.dw, p->R);
    if (persistent_variant(cfg.variant)) {
      const int rc2 = launch_persistent(p, a, rows, cfg, G, mv, sh.smem_bytes, st, &e);
      if (rc2 != GIRIH_OK) return rc2;
    }
    for (int64_t rho = 0; rho < rows && e == cudaSuccess && !persistent_variant(cfg.variant); ++rho) {
      int64_t a_min = 0, nd = 0;
      mwd_row_span(rho, cfg.dw, p->ny, &a_min, &nd);
      if (nd == 0) continue;
      a.rho = (int32_t)rho;
      a.a_min = (int32_t)a_min;
      e = launch_mwd_row(p->stencil, p->dtype, a, (int)nd, cfg.threads, G, mv, sh.smem_bytes, st);
    }
  }
  if (e == cudaSuccess && T % 2 == 1) e = launch_swap(u, u_prev, p->gstride * p->elem, st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GIRIH_OK;
}

// FED_PERSISTENT: build the FIFO of diamonds (row-major) and the per-row table, reset the FIFO
// counter, bump the epoch (flags of earlier sweeps never equal it) and launch as many clusters
// as the device holds at once (all resident, so dependency waits cannot deadlock).
// OVERLAP_PERSISTENT with zseg > 0: the items are (diamond, z segment); item (rho, a, j) waits
// for (rho, a, j-1) and for segment min(j + delta_rho, nseg - 1) of the two parents, so the FIFO
// orders them by j + (max delta + 1) rho (every dependency comes earlier), then by row and diamond.
static int launch_persistent(Plan* p, MwdArgs a, int64_t rows, const girih_config& cfg, int G, int mv,
                             int64_t smem, cudaStream_t st, cudaError_t* e_out) {
  const int zs = cfg.zseg > 0 && cfg.zseg < p->nz ? cfg.zseg : 0;
  const int nseg = zs ? (int)((p->nz + zs - 1) / zs) : 1;
  const int Hh = cfg.dw / p->R / 2, K = p->R + cfg.nf;
  int dmax = 0;
  for (int64_t rho = 1; rho < rows && zs; ++rho) {
    const int64_t d = std::max<int64_t>((rho - 1) * Hh + 1, 0) - std::max<int64_t>((rho - 2) * Hh + 1, 0);
    dmax = std::max(dmax, (int)(((d - 1) * K + p->R + zs - 1) / zs));
  }
  struct Item {
    int64_t key;
    int rho, a, seg;
  };
  std::vector<Item> order;
  std::vector<int> table;
  int64_t n_flags = 0;
  for (int64_t rho = 0; rho < rows; ++rho) {
    int64_t a_min = 0, nd = 0;
    mwd_row_span(rho, cfg.dw, p->ny, &a_min, &nd);
    table.push_back((int)n_flags);
    table.push_back((int)a_min);
    table.push_back((int)nd);
    n_flags += nd * nseg;
    for (int j = 0; j < nseg; ++j)
      for (int64_t k = 0; k < nd; ++k) order.push_back({j + (int64_t)(dmax + 1) * rho, (int)rho, (int)(a_min + k), j});
  }
  std::stable_sort(order.begin(), order.end(), [](const Item& x, const Item& y) {
    return x.key != y.key ? x.key < y.key : (x.rho != y.rho ? x.rho < y.rho : x.a < y.a);
  });
  std::vector<int> items, segs;
  for (const Item& it : order) {
    items.push_back(it.rho);
    items.push_back(it.a);
    segs.push_back(it.seg);
  }
  const int64_t n_items = (int64_t)order.size();
  *e_out = cudaSuccess;
  if (n_items == 0) return GIRIH_OK;
  std::vector<int> host(items);
  host.insert(host.end(), table.begin(), table.end());
  if (nseg > 1) host.insert(host.end(), segs.begin(), segs.end());
  cudaError_t e = cudaSuccess;
  if ((int64_t)host.size() > p->sched_cap) {
    if (p->sched) cudaFree(p->sched);
    p->sched = nullptr;
    p->sched_cap = 0;
    e = cudaMalloc(&p->sched, host.size() * sizeof(int));
    if (e != cudaSuccess) return fail(GIRIH_ENOMEM, "schedule buffer: %s", cudaGetErrorString(e));
    p->sched_cap = (int64_t)host.size();
    p->sched_T = -1;
  }
  if (n_flags > p->flags_cap) {
    if (p->flags) cudaFree(p->flags);
    p->flags = nullptr;
    p->flags_cap = 0;
    e = cudaMalloc(&p->flags, n_flags * sizeof(int));
    if (e != cudaSuccess) return fail(GIRIH_ENOMEM, "flag buffer: %s", cudaGetErrorString(e));
    // cleared on the sweep's own stream, so the clear is ordered before the kernel on any stream
    // (a recycled allocation may still hold an epoch of an earlier plan)
    e = cudaMemsetAsync(p->flags, 0, n_flags * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "flag reset");
    p->flags_cap = n_flags;
    p->epoch = 0;
  }
  if (!p->fifo) {
    e = cudaMalloc(&p->fifo, sizeof(int));
    if (e != cudaSuccess) return fail(GIRIH_ENOMEM, "FIFO counter: %s", cudaGetErrorString(e));
  }
  // the list depends on (T, dw, zseg) only: upload it when they change (a pageable copy has
  // taken the host data when it returns, and is ordered before the launch on the stream)
  if (p->sched_T != rows || p->sched_dw != cfg.dw || p->sched_zs != zs) {
    e = cudaMemcpyAsync(p->sched, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "schedule upload");
    p->sched_T = rows;
    p->sched_dw = cfg.dw;
    p->sched_zs = zs;
  }
  e = cudaMemsetAsync(p->fifo, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "schedule upload");
  if (++p->epoch == 0x7fffffff) {  // wrap: clear the flags so that no stale one matches
    p->epoch = 1;
    e = cudaMemsetAsync(p->flags, 0, p->flags_cap * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "flag reset");
  }
  int max_clusters = 0;
  e = mwd_prepare(p->stencil, p->dtype, cfg.cluster, cfg.threads, G, mv, smem, &max_clusters);
  if (e != cudaSuccess) return cuda_fail(e, "persistent launch configuration");
  if (max_clusters < 1) return fail(GIRIH_EINVAL, "no cluster of the configuration fits the device");
  a.persist = 1;
  a.n_items = (int32_t)n_items;
  a.epoch = p->epoch;
  a.items = p->sched;
  a.rows = p->sched + 2 * n_items;
  a.zseg = zs;
  a.nseg = nseg;
  a.segs = nseg > 1 ? a.rows + 3 * rows : nullptr;
  a.flags = p->flags;
  a.fifo = p->fifo;
  a.rho = 0;
  a.a_min = 0;
  const int ngrid = (int)std::min<int64_t>(n_items, max_clusters);
  *e_out = launch_mwd_row(p->stencil, p->dtype, a, ngrid, cfg.threads, G, mv, smem, st);
  return GIRIH_OK;
}

static const double kConst7[5] = {0.4, 0.1, 0, 0, 0};
static const double kConst25[5] = {-0.9, 0.05, 0.025, 0.0125, 0.00625};
static const double kConstBox[5] = {0.4, 0.05, 0.02, 0.0075, 0};
static const double kConstRB[5] = {0.0, 1.0 / 6.0, 0, 0, 0};

int validate_run(Plan* p, void* u, void* u_prev, const void* coeffs, const girih_params* params,
                 const double** c, const girih_config** cfg) {
  if (!p) return fail(GIRIH_EINVAL, "plan is NULL");
  if (!u || !u_prev) return fail(GIRIH_EINVAL, "u and u_prev must be non-NULL");
  if (u == u_prev) return fail(GIRIH_EINVAL, "u and u_prev must be distinct buffers");
  const uintptr_t mis = (reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev)) % p->elem;
  if (mis) return fail(GIRIH_EINVAL, "buffers must be %d-byte aligned", p->elem);
  const int nc = ncoef_of(p->stencil);
  if (nc > 0) {
    if (!coeffs) return fail(GIRIH_EINVAL, "stencil %d needs %d coefficient grids", p->stencil, nc);
    if (reinterpret_cast<uintptr_t>(coeffs) % p->elem) return fail(GIRIH_EINVAL, "coeffs misaligned");
  }
  const int64_t bytes = p->gstride * p->elem;
  const char* cu = static_cast<const char*>(u);
  const char* cp = static_cast<const char*>(u_prev);
  if (cu < cp + bytes && cp < cu + bytes) return fail(GIRIH_EINVAL, "u and u_prev overlap");
  *c = (params) ? params->c
                 : (is_box(p->stencil) ? kConstBox
                                       : (p->stencil == GIRIH_7PT_RBGS ? kConstRB
                                                                       : (radius_of(p->stencil) == 4 ? kConst25 : kConst7)));
  *cfg = (params && params->force_cfg) ? &params->cfg : &p->cfg;
  if ((*cfg)->algo == GIRIH_ALGO_MWD) {
    const bool ptrs16 = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev)) & 15) == 0;
    const int rc = check_config(p, *cfg, nullptr, nullptr, nullptr, nullptr, ptrs16);
    if (rc != GIRIH_OK) return rc;
    if ((*cfg)->variant == GIRIH_FED_BULK &&
        ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev)) & 15) != 0)
      return fail(GIRIH_EINVAL, "FED_BULK needs 16-byte aligned buffers");
    if (tma_variant((*cfg)->variant) && nc > 0 && (reinterpret_cast<uintptr_t>(coeffs) & 15) != 0)
      return fail(GIRIH_EINVAL, "%s reads coefficient grids in 16-byte vectors: coeffs must be 16-byte aligned",
                  variant_name((*cfg)->variant));
  } else if ((*cfg)->algo != GIRIH_ALGO_NAIVE) {
    return fail(GIRIH_EINVAL, "unknown algo %d", (*cfg)->algo);
  }
  return GIRIH_OK;
}

}  // namespace girih

using namespace girih;

extern "C" {

const char* girih_last_error(void) { return g_err.c_str(); }

int girih_plan(girih_plan_t* out, int32_t stencil, int64_t nx, int64_t ny, int64_t nz, int64_t ldx, int32_t dtype,
               int64_t T) {
  if (!out) return fail(GIRIH_EINVAL, "out is NULL");
  *out = nullptr;
  if (stencil < 0 || stencil > 6) return fail(GIRIH_EINVAL, "unknown stencil %d", stencil);
  if (dtype != GIRIH_F64 && dtype != GIRIH_F32) return fail(GIRIH_EINVAL, "unknown dtype %d", dtype);
  if (nx < 1 || ny < 1 || nz < 1) return fail(GIRIH_EINVAL, "sizes must be >= 1");
  if (T < 0 || T > (1LL << 30)) return fail(GIRIH_EINVAL, "T=%lld out of range", (long long)T);
  const int R = radius_of(stencil);
  if (ldx == 0) ldx = nx + 2 * R;
  if (ldx < nx + 2 * R) return fail(GIRIH_EINVAL, "ldx=%lld < nx + 2R", (long long)ldx);
  Plan* p = new (std::nothrow) Plan();
  if (!p) return fail(GIRIH_ENOMEM, "plan allocation failed");
  p->stencil = stencil;
  p->dtype = dtype;
  p->R = R;
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->ldx = ldx;
  p->T = T;
  p->elem = dtype == GIRIH_F64 ? 8 : 4;
  p->gstride = (nz + 2 * R) * (ny + 2 * R) * ldx;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  if (e != cudaSuccess) {
    delete p;
    cudaGetLastError();
    return cuda_fail(e, "device query");
  }
  p->smem_optin = optin;
  p->bulk_layout = (ldx * p->elem) % 16 == 0;
  e = cudaMalloc(&p->err, sizeof(int));
  // cleared and waited for here, so the word is zero before any stream of the caller uses it
  if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, sizeof(int), nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    delete p;
    cudaGetLastError();
    return fail(GIRIH_ENOMEM, "plan error word: %s", cudaGetErrorString(e));
  }
  p->cfg = default_config(p);
  *out = p;
  return GIRIH_OK;
}

int girih_plan_destroy(girih_plan_t plan) {
  if (!plan) return GIRIH_OK;
  Plan* p = plan;
  for (void* d : {p->host_u, p->host_up, p->host_co, p->tune_u, p->tune_up, p->tune_co, (void*)p->err,
                  (void*)p->sched, (void*)p->flags, (void*)p->fifo})
    if (d) cudaFree(d);
  delete p;
  return GIRIH_OK;
}

int girih_plan_get_config(girih_plan_t plan, girih_config* cfg) {
  if (!plan || !cfg) return fail(GIRIH_EINVAL, "NULL argument");
  *cfg = plan->cfg;
  return GIRIH_OK;
}

int girih_plan_set_config(girih_plan_t plan, const girih_config* cfg) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  const int rc = check_config(plan, cfg, nullptr, nullptr, nullptr);
  if (rc != GIRIH_OK) return rc;
  plan->cfg = *cfg;
  return GIRIH_OK;
}

int girih_config_check(girih_plan_t plan, const girih_config* cfg, int64_t* smem_bytes) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  return check_config(plan, cfg, smem_bytes, nullptr, nullptr);
}

int girih_plan_layout(girih_plan_t plan, int64_t* elems, int32_t* radius, int64_t* ldx) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  if (elems) *elems = plan->gstride;
  if (radius) *radius = plan->R;
  if (ldx) *ldx = plan->ldx;
  return GIRIH_OK;
}

int girih_plan_launch_count(girih_plan_t plan, const girih_config* cfg, int64_t* launches) {
  if (!plan || !launches) return fail(GIRIH_EINVAL, "NULL argument");
  const girih_config& c = cfg ? *cfg : plan->cfg;
  const int64_t T = plan->T;
  int64_t n = (c.algo == GIRIH_ALGO_NAIVE) ? T : mwd_rows(T, c.dw, plan->R);
  if (c.algo != GIRIH_ALGO_NAIVE && persistent_variant(c.variant) && T > 0) n = 1;
  if (T % 2 == 1) ++n;
  *launches = n;
  return GIRIH_OK;
}

int girih_run(girih_plan_t plan, void* u, void* u_prev, const void* coeffs, const girih_params* params,
              void* stream) {
  const double* c = nullptr;
  const girih_config* cfg = nullptr;
  int rc = validate_run(plan, u, u_prev, coeffs, params, &c, &cfg);
  if (rc != GIRIH_OK) return rc;
  if (plan->T == 0) return GIRIH_OK;
  return run_sweep(plan, plan->T, u, u_prev, coeffs, c, *cfg, static_cast<cudaStream_t>(stream));
}

int girih_status(girih_plan_t plan, void* stream) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int v = 0;
  e = cudaMemcpyAsync(&v, plan->err, sizeof(int), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  // cleared on the caller's stream: ordered before the plan's next sweep on that stream
  if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(plan->err, 0, sizeof(int), static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess && v != 0) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "reading the error word");
  if (v & GIRIH_ETIMEOUT) return fail(GIRIH_ETIMEOUT, "a bounded device wait ran out (a staged plane never arrived)");
  if (v) return fail(GIRIH_EKERNEL, "kernel error word %d", v);
  return GIRIH_OK;
}

int girih_run_host(girih_plan_t plan, void* u_host, void* u_prev_host, const void* coeffs_host,
                   const girih_params* params, void* stream) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  Plan* p = plan;
  if (!u_host || !u_prev_host) return fail(GIRIH_EINVAL, "host arrays must be non-NULL");
  const int nc = ncoef_of(p->stencil);
  if (nc > 0 && !coeffs_host) return fail(GIRIH_EINVAL, "coefficient grids missing");
  const size_t bytes = (size_t)(p->gstride * p->elem);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!p->host_u) e = cudaMalloc(&p->host_u, bytes);
  if (e == cudaSuccess && !p->host_up) e = cudaMalloc(&p->host_up, bytes);
  if (e == cudaSuccess && nc > 0 && !p->host_co) e = cudaMalloc(&p->host_co, bytes * nc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GIRIH_ENOMEM, "device buffers for host run: %s", cudaGetErrorString(e));
  }
  if (p->T == 0) return GIRIH_OK;  // nothing to advance (as girih_run)
  e = cudaMemcpyAsync(p->host_u, u_host, bytes, cudaMemcpyHostToDevice, st);
  // first-order stencils: u_prev is scratch whose halo equals u's, so it is made on the device
  if (e == cudaSuccess)
    e = second_order(p->stencil) ? cudaMemcpyAsync(p->host_up, u_prev_host, bytes, cudaMemcpyHostToDevice, st)
                                 : cudaMemcpyAsync(p->host_up, p->host_u, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && nc > 0) e = cudaMemcpyAsync(p->host_co, coeffs_host, bytes * nc, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
  int rc = girih_run(plan, p->host_u, p->host_up, nc > 0 ? p->host_co : nullptr, params, stream);
  if (rc != GIRIH_OK) return rc;
  e = cudaMemcpyAsync(u_host, p->host_u, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_prev_host, p->host_up, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
  return girih_status(plan, stream);
}

// Eq. 3 (general R; Eq. 2 for R = 1 is the same expression up to the paper's approximation):
// C_S = N_xb * [ N_D * D_w * (D_w/2 - R + N_F) + 2R (D_w + W_w) ],  W_w = D_w - 2R + N_F.
double girih_model_cache_block(double n_xb, int32_t dw, int32_t nf, int32_t r, int32_t nd) {
  const double ww = (double)dw - 2.0 * r + nf;
  return n_xb * ((double)nd * dw * ((double)dw / 2.0 - r + nf) + 2.0 * r * (dw + ww));
}

// Eq. 5 (Eq. 4 for R = 1): B_C = 2 s R [ (2 D_w - 2R) + (N_D D_w + 2R) ] / D_w^2 bytes/LUP,
// s = element size (the paper's 16R is 2 s R with s = 8).
double girih_model_code_balance(int32_t dw, int32_t r, int32_t nd, int32_t elem_bytes) {
  if (dw <= 0) return 0.0;
  const double d = dw;
  return 2.0 * elem_bytes * r * ((2.0 * d - 2.0 * r) + (nd * d + 2.0 * r)) / (d * d);
}

}  // extern "C"
