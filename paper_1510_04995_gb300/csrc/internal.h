// Internal interfaces between the C-ABI layer (api.cu, tuner.cu) and the kernel translation
// units (naive.cu, mwd.cu, mlp.cu).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/girih.h"

namespace girih {

// Geometry of one padded grid.
struct Grid {
  int64_t nx, ny, nz, ldx;  // interior sizes and leading dimension
  int64_t sy;               // ny + 2R (rows per plane)
  int64_t gstride;          // elements per grid: (nz+2R)*sy*ldx
};

// One naive time step (Sect. 2.1.1): U <- S(V) (and U's own old value for second order).
struct NaiveArgs {
  Grid g;
  const void* V;
  void* U;
  const void* coef;
  double c[5];
  float cf[5];  // the same constants rounded to FP32 (FP32 kernels read these: no conversion on device)
  int32_t zc;  // z planes per block
  int32_t v16;  // rows of 16-byte multiples and 16-byte aligned buffers: 16-byte staging
  int32_t t;    // the time step this launch makes (the red-black colour mask depends on it)
};
cudaError_t launch_naive_step(int stencil, int dtype, const NaiveArgs& a, cudaStream_t st);
// Resident blocks per SM of the naive kernel, and the z chunk (planes per block) that fills the
// device's block slots in whole waves best.
int naive_resident_blocks(int stencil, int dtype, bool v16);
int naive_tile_x(int stencil, int dtype, bool v16);  // tile columns of the naive kernel
int naive_tile_y(int stencil, int dtype);             // tile rows (threads per block = 16 * rows)
int naive_z_chunk(int64_t nx, int64_t ny, int64_t nz, int R, int tile_x, int tile_y, int resident_per_sm,
                  int sm_count);

// One row of diamonds of the multi-threaded wavefront-diamond sweep (Sect. 4.2.1).
struct MwdArgs {
  Grid g;
  void* buf0;        // global buffer holding even time levels (the caller's u)
  void* buf1;        // odd time levels (the caller's u_prev)
  const void* coef;
  double c[5];
  float cf[5];       // the same constants rounded to FP32
  int32_t T;         // total time steps of the sweep
  int32_t rho;       // diamond row index
  int32_t dw, nf, K, H;  // diamond width, wavefront width, level skew (R + nf), levels per diamond
  int32_t a_min;     // index of the first diamond of the row
  int32_t C, XW;     // blocks per tile (cluster) and x slab width per block
  int32_t NZ, YW, XT;  // shared ring: planes, rows, columns per buffer
  int* err;          // device error word: bounded waits that ran out set GIRIH_ETIMEOUT here
  int32_t relaxed;   // RELAXED variant: neighbour hand-off instead of the cluster barrier
  // persistent schedule (FED_PERSISTENT): diamonds (rho, a) in FIFO order, per row
  // (first item, a_min, count), completion flags (= epoch when done), the FIFO counter
  int32_t persist, n_items, epoch;
  const int* items;
  const int* rows;
  int* flags;
  int* fifo;
  // OVERLAP_PERSISTENT split along z: items are (rho, a, segment), segs[item] the segment;
  // segment j runs the tile's wavefront steps [j zseg, (j+1) zseg), the last one to the tile's
  // end; the flag of (rho, a, j) is rows[3 rho] + (a - a_min(rho)) nseg + j.  nseg = 1: whole
  // tiles (zseg and segs unused)
  int32_t zseg, nseg;
  const int* segs;
  int32_t lead;  // RELAXED_PERSISTENT: steps between a plane's staging and its first use (3..8)
  int32_t PE;    // RELAXED_PERSISTENT: elements per ring slot (YW * XT rounded up to 128 bytes)
  int32_t HMO;   // OVERLAP_PERSISTENT: staged columns on each side of the slab
  // RELAXED_PERSISTENT: 3D tensor maps of buf0 and buf1 (padded grid, box XT x YW x 1) for the
  // staging copies; the kernel takes MwdArgs as a __grid_constant__ parameter
  alignas(64) CUtensorMap tm[2];
};

struct MwdShape {
  int32_t NZ, YW, XT;
  int64_t smem_bytes;
  int32_t PE = 0;  // RELAXED_PERSISTENT: elements per ring slot
  int32_t HM = 0;  // OVERLAP_PERSISTENT: staged columns on each side of the slab
};
// Data paths of the blocked kernel: per-element staging (any layout); 16-byte vectors on a
// shifted slab partition (rows of 16-byte multiples, 16-byte aligned buffers) moved by cp.async
// and vector stores; or the same partition with whole rows moved by the bulk-copy (TMA) engine
// (FED_BULK).
// MV_ASYNC: the vector path's partition and data movement with neighbour-only synchronisation
// and the persistent schedule (RELAXED_PERSISTENT, mwd_async.cuh; radius-1 first-order stencils).
// MV_OVL: the same blocks on x slabs widened by the halo every level needs, with no exchange
// between blocks inside a step (OVERLAP_PERSISTENT, mwd_overlap.cuh).
// MV_OVLZ: MV_OVL with its tiles split along z (separate kernel instances, so that the whole-tile
// ones carry none of the segment logic).
enum { MV_ELEM = 0, MV_VEC = 1, MV_BULK = 2, MV_ASYNC = 3, MV_OVL = 4, MV_OVLZ = 5 };
inline bool mv_ovl(int mv) { return mv == MV_OVL || mv == MV_OVLZ; }
inline bool mv_tma(int mv) { return mv == MV_ASYNC || mv_ovl(mv); }
// OVERLAP_PERSISTENT: staged columns on each side of a slab, (H - 1) R rounded up to 16 bytes
// (the bottom level of an unclipped diamond reads (smax + 1) R = (H - 1) R columns beyond it).
inline int ovl_margin(int H, int R, int a16) { return ((H - 1) * R + a16 - 1) / a16 * a16; }
// Its tasks (row pair x vx columns over the widened level ranges) for an unclipped diamond on an
// interior slab of XW columns (a16: elements per 16 bytes, the margin's rounding).
int64_t mwd_ovl_tasks(int R, int dw, int XW, int vx, int a16);
// stencils the RELAXED_PERSISTENT kernel is built for
// stencils the OVERLAP_PERSISTENT kernel is built for: those and the radius-4 ones
inline bool ovl_stencil(int stencil) {
  return stencil == GIRIH_7PT_CONST || stencil == GIRIH_7PT_VAR || stencil == GIRIH_7PT_RBGS ||
         stencil == GIRIH_25PT_CONST || stencil == GIRIH_25PT_VAR || stencil == GIRIH_25PT_CGRID;
}
inline bool async_stencil(int stencil) {
  return stencil == GIRIH_7PT_CONST || stencil == GIRIH_7PT_VAR || stencil == GIRIH_7PT_RBGS;
}
// Staging lead (steps) of the RELAXED_PERSISTENT kernel: the host takes the deepest lead in
// [kAsyncLeadMin, kAsyncLeadMax] whose ring still fits as many blocks per SM as the shallowest.
#ifndef GIRIH_ASYNC_LEAD_MAX
#define GIRIH_ASYNC_LEAD_MAX 8
#endif
constexpr int kAsyncLeadMin = 3;
constexpr int kAsyncMovers = 32;    // threads of the RELAXED_PERSISTENT block that move data
constexpr int kOvlMovers = 64;      // of the OVERLAP_PERSISTENT block (a staging and a waiting warp)
constexpr int kAsyncLoadBars = 8;   // its staging mbarriers (the lead is at most 8)
constexpr int kAsyncLeadMax = GIRIH_ASYNC_LEAD_MAX;
// Largest block of the warp-specialised kernels for G tasks per thread (their launch bound); the
// variable-coefficient stencils hold a prefetched plane of coefficients per task in registers,
// the radius-4 tasks (OVERLAP_PERSISTENT) windows of 2R+1 planes.
constexpr int async_max_threads(int G, bool coef, bool r4 = false) {
  if (r4) return G == 1 ? 512 : (G == 2 ? 320 : 160);  // radius 4: windows of 2R+1 planes
  return coef ? (G == 1 ? 512 : (G == 2 ? 288 : 160)) : (G == 1 ? 640 : (G == 2 ? 512 : 256));
}
inline bool mv_shifted(int mv) { return mv != MV_ELEM; }
MwdShape mwd_shape(int stencil, int dtype, int dw, int nf, int XW, int mv, int lead = kAsyncLeadMin);
// RELAXED_PERSISTENT: the staging lead for a configuration (see kAsyncLeadMax) and its shape.
int mwd_async_lead(int stencil, int dtype, int dw, int nf, int XW, int threads, int G, int64_t smem_optin,
                   int mv = MV_ASYNC);
// Launch one diamond row: ndiam tiles, each a cluster of a.C blocks of `threads` threads.
// G = groups per thread (1, 2, 4 or 8), from mwd_pairs_per_thread; mv = data path.
cudaError_t launch_mwd_row(int stencil, int dtype, const MwdArgs& a, int ndiam, int threads, int G, int mv,
                           int64_t smem, cudaStream_t st);
// Configure kernel attributes (dynamic shared memory, non-portable clusters); returns the max
// active clusters the device reports for the configuration (0 = cannot be scheduled).
cudaError_t mwd_prepare(int stencil, int dtype, int C, int threads, int G, int mv, int64_t smem, int* max_clusters);
int mwd_max_pairs(int R, int dw);
int mwd_pairs_per_thread(int stencil, int dtype, int dw, int XW, int threads, int mv);
// Columns per group of the blocked kernel and its launch-bound divisor (mirror the device side).
inline int radius_of(int stencil) { return (stencil >= 2 && stencil <= 4) ? 4 : 1; }
inline int ncoef_of(int stencil) { return stencil == 1 ? 7 : (stencil == 3 ? 13 : (stencil == 4 ? 1 : 0)); }
inline bool is_box(int stencil) { return stencil == GIRIH_27PT_BOX; }
// stencils whose blocked sweep exists on the 16-byte vector path only
inline bool vec_only(int stencil) { return stencil == GIRIH_27PT_BOX || stencil == GIRIH_7PT_RBGS; }
inline bool second_order(int stencil) { return stencil >= 2 && stencil <= 4; }
inline int mwd_vx(int stencil, int dtype, int mv) {
  const bool r1 = radius_of(stencil) == 1;
  if (mv_ovl(mv) && r1 && dtype == GIRIH_F64 && ncoef_of(stencil) == 0) return 1;
  if (mv_shifted(mv)) return r1 ? (dtype == GIRIH_F64 ? 2 : 4) : (dtype == GIRIH_F32 ? 2 : 1);
  return (!r1 && dtype == GIRIH_F64) ? 1 : (dtype == GIRIH_F64 ? 2 : 4);
}
inline int mwd_lbf(int stencil, int dtype, int mv) {
  const bool r1 = radius_of(stencil) == 1;
  if (mv_shifted(mv)) return (r1 && !is_box(stencil)) ? 2 : 4;
  return mwd_vx(stencil, dtype, mv) == 1 ? 1 : (r1 ? 2 : 4);
}
// Largest block for G groups per thread (the kernel's launch bound).
inline int mwd_max_threads(int G, int lbf) {
  const int t = 1024 / (G * lbf);
  return t > 1024 ? 1024 : t;
}
// Planes are staged this many wavefront steps ahead of use (cp.async paths / bulk-copy path).
// A cp.async group committed at step k is waited for (wait_group PD-2) before the barrier that
// ends step k+PD-1, so it has PD-1 steps to land.
#define MWD_PREFETCH 3
#define MWD_PREFETCH_BULK 3
// Extra ring planes per wavefront width, so that a slot is restaged only after every write-back
// that may still read it: cp.async paths -- the previous step's write-back, which threads of the
// block that have not yet passed that step's barrier may still be doing; bulk-copy path -- the
// write-back copies of the two previous steps.
#define MWD_PLAIN_SLACK 1
#define MWD_BULK_SLACK 2


// In-place exchange of two device arrays (odd T puts level T back into u).
cudaError_t launch_swap(void* a, void* b, int64_t bytes, cudaStream_t st);


}  // namespace girih
