/*
 * girih.h -- C ABI of the GB300 (sm_103a) temporally blocked stencil sweep library.
 *
 * The library advances a 3D grid by T time steps of one of seven Jacobi-style stencils
 * (Malas, Hager, Ltaief, Keyes, "Multi-dimensional intra-tile parallelization for
 * memory-starved stencil computations", arXiv 1510.04995):
 *   GIRIH_7PT_CONST  Listing 1: first order in time, radius 1, constants c0, c1.
 *   GIRIH_7PT_VAR    Listing 2: first order in time, radius 1, 7 coefficient grids.
 *   GIRIH_25PT_CONST Listing 3 with the per-point factor fixed to 1: second order in time
 *                    (U = 2V - U + ...), radius 4, constants c0..c4.
 *   GIRIH_25PT_VAR   Listing 4's 13 axis-symmetric coefficient grids, second order in time.
 *   GIRIH_25PT_CGRID Listing 3 as printed: second order in time, radius 4, constants c0..c4
 *                    and one per-point factor grid C multiplying the bracket (U = 2V - U +
 *                    C*(c0*V + sum_r c_r*pairs_r)); three domain-sized streams (Sect. 3.5).
 *   GIRIH_27PT_BOX   the box-shaped operator of Sect. 8.4: first order in time, radius 1, all 26
 *                    neighbours at Chebyshev distance 1, constants c0 (centre), c1 (the 6 face
 *                    neighbours), c2 (the 12 edge neighbours), c3 (the 8 corner neighbours).
 *                    Its blocked sweep runs on the 16-byte vector path only (rows of 16-byte
 *                    multiples, 16-byte aligned buffers); the naive sweep takes any layout.
 *   GIRIH_7PT_RBGS   red-black Gauss-Seidel on the 7-point constant operator (Sect. 8.4): time
 *                    step t is a half-sweep updating the points whose interior coordinates have
 *                    x + y + z + t even (c0*V + c1*(neighbour pairs)) and keeping the others;
 *                    T = 2 x the red-black iterations.  Computed in the two-buffer form (the
 *                    kept colour is copied), bit for bit the in-place sweep.  Blocked sweep on
 *                    the vector path only, as for 27PT_BOX.
 * Two algorithms reach the same result (Sect. 2.1): the naive sweep (one pass over the grid per
 * time step, Sect. 2.1.1) and the multi-threaded wavefront-diamond sweep (MWD, Sect. 4.2.1):
 * diamond tiles along y (Sect. 2.1.2), a wavefront along z, several time steps per pass over
 * memory, one tile shared by a cluster of thread blocks (the paper's thread group, Sect. 4.1).
 *
 * Conventions for every function:
 *  - Return value: GIRIH_OK (0) or one of the GIRIH_E* codes below.  On failure a message is
 *    available from girih_last_error() (thread-local, valid until the next call on that thread).
 *  - Device pointers are raw CUDA device addresses owned by the caller; the library never frees
 *    them.  Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Grid layout ("padded layout"): element (i, j, k) with 0 <= i < ldx, 0 <= j < ny+2R,
 *    0 <= k < nz+2R lives at offset (k*(ny+2R) + j)*ldx + i, x fastest.  The interior is
 *    i in [R, R+nx), j in [R, R+ny), k in [R, R+nz); the R-wide halo is read, never written
 *    (the listings' loops start at R and stop R before the end).  ldx >= nx + 2R is the leading
 *    dimension (Sect. 4.2.3 pads the leading dimension); 0 means dense (nx + 2R).
 */
#ifndef GIRIH_H
#define GIRIH_H

#include <stdint.h>

#if defined(__GNUC__)
#define GIRIH_API __attribute__((visibility("default")))
#else
#define GIRIH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- enums and status codes -------------------------------------------------------------- */
typedef enum {
  GIRIH_7PT_CONST = 0,
  GIRIH_7PT_VAR = 1,
  GIRIH_25PT_CONST = 2,
  GIRIH_25PT_VAR = 3,
  GIRIH_25PT_CGRID = 4,
  GIRIH_27PT_BOX = 5,
  GIRIH_7PT_RBGS = 6
} girih_stencil;
typedef enum { GIRIH_F64 = 0, GIRIH_F32 = 1 } girih_dtype;
typedef enum { GIRIH_ALGO_NAIVE = 0, GIRIH_ALGO_MWD = 1 } girih_algo;
/* Wavefront synchronisation variants of Sect. 4.2.1:
 *   FED     -- fixed execution to data: each thread block of the cluster always updates the
 *              same x slab of the tile; one cluster-wide barrier per wavefront step.  Planes
 *              move in 16-byte chunks (cp.async in, vector stores out) when ldx*elem is a
 *              multiple of 16 bytes and the buffers are 16-byte aligned, else element by
 *              element (any layout).
 *   FED_BULK -- FED with whole rows moved by the bulk-copy (TMA) engine, issued by one warp
 *              between the halves of each step's barrier; needs ldx*elem to be a multiple of
 *              16 bytes, 16-byte aligned buffers and planes of fewer than 2^30 elements.
 *   RELAXED -- no cluster-wide barrier: each block of the cluster publishes its completed
 *              wavefront steps to its two x neighbours (progress counters in their shared
 *              memory, release/acquire at cluster scope) and waits only for theirs, the
 *              neighbour hand-off of the paper's relaxed synchronisation.  Data movement as
 *              FED; with a cluster of one block it is the same as FED.
 *   FED_ELEM, RELAXED_ELEM -- FED and RELAXED forced onto the element-by-element path on any
 *              layout (the tuner weighs both data paths).
 *   FED_PERSISTENT -- FED on the vector path with the FIFO runtime of Sect. 4.2.3: one launch
 *              per sweep, clusters take diamonds in row-major order and start each once the
 *              two diamonds of the previous row it depends on have completed (bounded waits
 *              on per-diamond flags).  Needs the vector path's layout (16-byte rows, 16-byte
 *              aligned buffers).  The plan owns the diamond list, the flags and the FIFO
 *              counter (allocated on first use, freed by girih_plan_destroy), so sweeps of one
 *              plan must not run concurrently on different streams.  A wait that runs out
 *              (2 s) makes girih_status return GIRIH_ETIMEOUT.
 *   RELAXED_PERSISTENT -- the persistent FIFO schedule of FED_PERSISTENT with the relaxed
 *              synchronisation of Sect. 4.2.1 instead of a cluster barrier per wavefront step:
 *              a block waits, per step, for its own results (block barrier) and for exactly the
 *              x-halo bytes its two neighbours computed in that step, which they store into its
 *              shared memory asynchronously (st.async, counted on an mbarrier).  Radius-1
 *              first-order stencils (7PT_CONST, 7PT_VAR, 7PT_RBGS) on the vector path's
 *              layout (16-byte rows, 16-byte aligned buffers and coefficient grids); EINVAL
 *              otherwise.  Buffers and bounded waits as FED_PERSISTENT.
 *   OVERLAP_PERSISTENT -- RELAXED_PERSISTENT's schedule, blocks and data movement with no
 *              exchange between the blocks of a cluster inside a wavefront step: each block
 *              stages its x slab plus (H-1)R columns per side (rounded up to 16 bytes) and
 *              updates level s of the diamond over its slab widened by (H-2-s)R columns per
 *              side, repeating the neighbours' edge columns instead of receiving them (the
 *              results stay bit-identical).  Before storing final values a block checks that
 *              both neighbours have staged the planes concerned (progress words in shared
 *              memory at cluster scope; a bounded wait).  One staging and one waiting warp
 *              (blocks of more than 64 threads).  Built for the 7-point, red-black and
 *              25-point stencils (not the box stencil; EINVAL); layout, alignment and nf = 1
 *              rules as RELAXED_PERSISTENT.  With girih_config.zseg > 0 each diamond is split
 *              along z into segments scheduled as separate items (bounded waits on the
 *              segments' completion flags, as on the diamonds').                           */
typedef enum {
  GIRIH_FED = 0,
  GIRIH_RELAXED = 1,
  GIRIH_FED_BULK = 2,
  GIRIH_FED_ELEM = 3,
  GIRIH_RELAXED_ELEM = 4,
  GIRIH_FED_PERSISTENT = 5,
  GIRIH_RELAXED_PERSISTENT = 6,
  GIRIH_OVERLAP_PERSISTENT = 7
} girih_variant;

#define GIRIH_OK 0
#define GIRIH_EINVAL 1   /* bad enum, size, T, pointer, alignment, or config: nothing enqueued */
#define GIRIH_ENOMEM 2   /* a host or device allocation failed                                 */
#define GIRIH_ECUDA 3    /* a CUDA call failed (message has the CUDA error string)             */
#define GIRIH_EKERNEL 4  /* a kernel's own consistency check fired                             */
#define GIRIH_ETIMEOUT 5 /* a bounded device-side wait ran out                                 */
#define GIRIH_ENOTIMPL 6 /* the combination is not available                                   */

/* Tunable parameters of the blocked sweep (Sect. 4.2.2 tunes diamond width, wavefront width
 * and the thread-group shape).  Fields:
 *   algo     GIRIH_ALGO_NAIVE or GIRIH_ALGO_MWD.
 *   dw       diamond width D_w along y (a multiple of 2R, >= 2R); MWD only.
 *   nf       wavefront tile width N_F: z planes each time level advances per step (1..4).
 *   cluster  thread blocks sharing one tile along x (1, 2, 4, 8 or 16).
 *   threads  threads per block (multiple of 32, 64..1024).
 *   variant  girih_variant.
 *   zseg     OVERLAP_PERSISTENT only (0 elsewhere): the parallelepiped split of an extruded
 *            diamond along z (Sect. 8).  0 = whole tiles.  zseg >= 1: segment j of a tile runs
 *            the tile's wavefront steps [j zseg, (j+1) zseg) -- the last segment runs to the
 *            tile's end -- as its own item of the persistent schedule, so that a diamond of the
 *            next row starts on its first planes while this one still works on its later ones
 *            (concurrency for grids with few diamonds per row).  A segment starts once its
 *            tile's previous segment and, in the two parent diamonds, the segments up to
 *            j + ceil(((tb - tb_parent - 1) K + R) / zseg) have completed (tb: first level,
 *            K = R + nf); values cross segments through global memory (each segment but the
 *            last also stores the values of its last K + R steps, 2K for the second-order
 *            stencils).  EINVAL: zseg < 0, or zseg > 0 with another variant.              */
typedef struct girih_config {
  int32_t algo;
  int32_t dw;
  int32_t nf;
  int32_t cluster;
  int32_t threads;
  int32_t variant;
  int32_t zseg;
} girih_config;

/* Per-call parameters.  c[] holds the constant coefficients: 7PT_CONST uses c[0]=c0 (centre),
 * c[1]=c1 (the six neighbours); 25PT_CONST and 25PT_CGRID use c[0] (centre) and c[r] for the six
 * neighbours at distance r = 1..4; 27PT_BOX uses c[0] (centre), c[1] (faces), c[2] (edges) and
 * c[3] (corners); 7PT_RBGS c[0] and c[1] like 7PT_CONST.  Ignored by the variable-coefficient stencils.  If force_cfg is non-zero,
 * cfg replaces the plan's configuration for this call.                                     */
typedef struct girih_params {
  double c[5];
  int32_t force_cfg;
  girih_config cfg;
} girih_params;

typedef struct girih_plan_s* girih_plan_t;

/* ---- plan / run ---------------------------------------------------------------------------- */

/* Create a plan for T steps of `stencil` on an nx*ny*nz interior (halo R implied: 1 for the
 * 7-point, box and red-black stencils, 4 for the 25-point ones) in `dtype`, leading dimension ldx (0 = dense).
 * Queries the current device and picks a default configuration (largest feasible diamond).
 * Writes *out = NULL on failure.  EINVAL: bad enum, nx/ny/nz < 1, T < 0, ldx < nx + 2R.    */
GIRIH_API int girih_plan(girih_plan_t* out, int32_t stencil, int64_t nx, int64_t ny, int64_t nz, int64_t ldx,
               int32_t dtype, int64_t T);

/* Release a plan (NULL is accepted). */
GIRIH_API int girih_plan_destroy(girih_plan_t plan);

/* Read or replace the plan's configuration.  girih_plan_set_config returns EINVAL (and leaves
 * the plan unchanged) if the configuration is not feasible on this device for this problem.  */
GIRIH_API int girih_plan_get_config(girih_plan_t plan, girih_config* cfg);
GIRIH_API int girih_plan_set_config(girih_plan_t plan, const girih_config* cfg);

/* Feasibility of a configuration for the plan's problem on the current device: GIRIH_OK or
 * EINVAL.  If smem_bytes is not NULL it receives the shared memory one block needs.            */
GIRIH_API int girih_config_check(girih_plan_t plan, const girih_config* cfg, int64_t* smem_bytes);

/* Advance the grids by the plan's T steps, asynchronously on `stream`.
 *   u       device buffer with level 0 (u^0); on return level T.
 *   u_prev  device buffer: for the second-order stencils level -1 on entry and level T-1 on
 *           return; for the first-order stencils scratch whose halo must equal u's halo (on
 *           return it holds level T-1, or is unchanged when T = 0).
 *   coeffs  NULL for 7PT_CONST, 25PT_CONST, 27PT_BOX and 7PT_RBGS; else 7 (7PT_VAR: C0 centre, C1 x+1, C2 x-1,
 *           C3 y+1, C4 y-1, C5 z+1, C6 z-1; Listing 2), 13 (25PT_VAR: C00 centre, then for
 *           r = 1..4 the x, y, z pairs at distance r; Listing 4) or 1 (25PT_CGRID: the factor C
 *           of Listing 3) grids of the padded layout, back to back; their halo cells are never
 *           read.
 *   params  coefficients and optional forced configuration (NULL: 7PT_CONST uses the workload
 *           constants c0=0.4, c1=0.1; 25PT_CONST and 25PT_CGRID c0=-0.9, c_r=0.1/2^r; 27PT_BOX
 *           0.4, 0.05, 0.02, 0.0075; 7PT_RBGS c0=0, c1=1/6, the Laplace equation).
 * Pointers must be 8-byte (F64) or 4-byte (F32) aligned (16-byte for GIRIH_FED_BULK) and
 * u != u_prev.  The two buffers'
 * roles alternate every step (Listing 3's pointer swap); for odd T one in-place exchange kernel
 * puts level T back into u.  EINVAL leaves the buffers untouched and enqueues nothing.       */
GIRIH_API int girih_run(girih_plan_t plan, void* u, void* u_prev, const void* coeffs, const girih_params* params,
              void* stream);

/* Convenience for callers holding HOST arrays (pinned or pageable): copies u, u_prev and coeffs
 * to device buffers the plan owns (allocated on first use, freed by girih_plan_destroy), runs
 * girih_run on `stream`, copies u and u_prev back, and synchronises the stream.  For the
 * first-order stencils u_prev_host is not read: its device copy is made from u on the device
 * (the scratch buffer's halo must equal u's), which saves one host-to-device transfer.  T = 0
 * copies nothing and leaves both host arrays as they are.                                     */
GIRIH_API int girih_run_host(girih_plan_t plan, void* u_host, void* u_prev_host, const void* coeffs_host,
                   const girih_params* params, void* stream);

/* Synchronise `stream` and report device-side failures of the plan's previous runs: GIRIH_OK,
 * GIRIH_ETIMEOUT (a bounded wait of the blocked kernel ran out; the results are not valid) or
 * GIRIH_EKERNEL.  Clears the plan's error word.  girih_run_host calls it itself.            */
GIRIH_API int girih_status(girih_plan_t plan, void* stream);

/* Failure-path check of the device-side bounded waits (no counterpart in the paper; Sect. 4.2.1's
 * relaxed synchronisation is the wait being checked): enqueues on `stream` one block that runs
 * the RELAXED neighbour wait on progress counters nothing advances, limited to limit_ns
 * nanoseconds of the GPU's global timer (1e3 .. 2e9).  The wait gives up and sets the plan's
 * error word, so a following girih_status returns GIRIH_ETIMEOUT; the context stays usable.
 * Returns GIRIH_EINVAL for a NULL plan or a limit outside the range (nothing enqueued), or
 * GIRIH_ECUDA if the launch fails.                                                          */
GIRIH_API int girih_check_bounded_wait(girih_plan_t plan, int64_t limit_ns, void* stream);

/* Measured fused multiply-add throughput of the current GPU in `dtype` (no counterpart in the
 * paper: it is the denominator of the arithmetic roofline of the FP64 sweeps, which this GPU's
 * FP64 pipe bounds before HBM does).  Runs eight independent FMA chains per thread on every SM
 * (a short calibration launch, then one of about 0.1 s) on `stream`, synchronises it, and writes
 * the rate in FMA instructions per second (thread level; 2 flops each) to *fma_per_s and the
 * timed launch's duration to *seconds (may be NULL).  Allocates and frees a small device
 * buffer.  EINVAL for a NULL fma_per_s or an unknown dtype; ECUDA if a launch fails.          */
GIRIH_API int girih_measure_fma_rate(int32_t dtype, double* fma_per_s, double* seconds, void* stream);

/* Elements of one padded grid for the plan ((nz+2R)*(ny+2R)*ldx) and the halo width R. */
GIRIH_API int girih_plan_layout(girih_plan_t plan, int64_t* elems_per_grid, int32_t* radius, int64_t* ldx);

/* Number of kernel launches girih_run enqueues with the given configuration (NULL = plan's). */
GIRIH_API int girih_plan_launch_count(girih_plan_t plan, const girih_config* cfg, int64_t* launches);

GIRIH_API const char* girih_last_error(void);

/* ---- models of Sect. 3.3 / 3.4 ------------------------------------------------------------- */

/* Cache block size C_S in bytes of one wavefront-diamond tile (Eq. 3; for R = 1 this is the
 * paper's Eq. 2 up to the paper's own approximation): n_xb = bytes of the tile's leading
 * dimension, dw = diamond width, nf = wavefront width, r = radius, nd = domain-sized streams.  */
GIRIH_API double girih_model_cache_block(double n_xb, int32_t dw, int32_t nf, int32_t r, int32_t nd);

/* Code balance B_C in bytes per lattice-site update of the blocked sweep (Eq. 5; Eq. 4 for
 * R = 1) for elements of `elem_bytes` bytes (8: the paper's 16R factor; 4: 8R).             */
GIRIH_API double girih_model_code_balance(int32_t dw, int32_t r, int32_t nd, int32_t elem_bytes);

/* ---- auto-tuner (Sect. 4.2.2) ---------------------------------------------------------------- */

/* One timing row of the tuner's database. */
typedef struct girih_tune_row {
  girih_config cfg;
  double glups;      /* giga lattice-site updates per second, at the accepted test length */
  double seconds;    /* time of that accepted measurement                                  */
  int64_t steps;     /* time steps of the accepted measurement                             */
  int64_t smem;      /* shared memory per block                                            */
  double tune_seconds; /* host wall time spent measuring this candidate (all test lengths) */
} girih_tune_row;

/* Enumerate the candidate configurations (naive sweep plus every MWD diamond width, wavefront
 * width, cluster size and thread count) for the plan's problem; infeasible ones (shared memory
 * above the device limit, per the cache-block model of Eq. 3, or an unschedulable cluster) are
 * dropped.  Writes up to `cap` configurations and returns their number in *count.             */
GIRIH_API int girih_tune_candidates(girih_plan_t plan, girih_config* out, int32_t cap, int32_t* count);

/* Time one configuration the way Sect. 4.2.2 does: on tuner-owned device arrays, with a test
 * length that grows in whole diamond rows until two consecutive measurements agree within
 * `tol` (relative) or max_steps is reached.  Fills *row.                                       */
GIRIH_API int girih_tune_measure(girih_plan_t plan, const girih_config* cfg, double tol, int64_t max_steps,
                       girih_tune_row* row);

/* Exhaustive tuning: measure every candidate (the given list of n_cands configurations, or all of
 * girih_tune_candidates when cands is NULL), append one CSV line per candidate to db_path (NULL:
 * no file), set the plan's configuration to the fastest and return it in *best.  CSV columns:
 * stencil, dtype, nx, ny, nz, algo, dw, nf, cluster, threads, variant, glups, seconds, steps,
 * smem, tune_seconds.  Infeasible listed candidates return EINVAL before anything is measured. */
GIRIH_API int girih_tune_exhaustive(girih_plan_t plan, const girih_config* cands, int32_t n_cands, double tol,
                                    int64_t max_steps, const char* db_path, girih_tune_row* best, int32_t* n_measured);

/* ---- learned tuner: 3-layer MLP (D -> 64 -> 64 -> 1, ReLU), FP32, CUDA kernels --------------- */

/* Features of a configuration for the network (writes GIRIH_MLP_FEATURES floats): stencil
 * one-hot in [0, 4) (25PT_CGRID shares the 25PT_CONST slot, its third stream showing in the
 * model code balance, feature 14; 27PT_BOX and 7PT_RBGS share the 7PT_CONST slot), dtype, log sizes, algorithm, diamond width, wavefront width,
 * cluster, threads, variant, log code balance, log slab width.                                */
#define GIRIH_MLP_FEATURES 16
#define GIRIH_MLP_HIDDEN 64
GIRIH_API int girih_mlp_features(int32_t stencil, int32_t dtype, int64_t nx, int64_t ny, int64_t nz,
                       const girih_config* cfg, float* out);

/* Number of parameters for input width d: 64d + 64 + 64*64 + 64 + 64 + 1, laid out as
 * [W1 (64 x d row-major), b1, W2 (64 x 64), b2, W3 (1 x 64), b3].                            */
GIRIH_API int64_t girih_mlp_num_params(int32_t d);

/* Forward pass on device arrays: y[n] = net(X[n x d]).  workspace: device scratch of at least
 * girih_mlp_workspace_floats(n) floats.                                                        */
GIRIH_API int64_t girih_mlp_workspace_floats(int32_t n);
GIRIH_API int girih_mlp_forward(const float* params, const float* X, int32_t n, int32_t d, float* y, float* workspace,
                      void* stream);

/* Gradient of the mean squared error (1/n) sum (y - t)^2 with respect to the parameters, on
 * device: grad has girih_mlp_num_params(d) floats; loss (device, 1 float) may be NULL.         */
GIRIH_API int girih_mlp_backward(const float* params, const float* X, const float* t, int32_t n, int32_t d, float* grad,
                       float* loss, float* workspace, void* stream);

/* Allocation-free variant of girih_mlp_backward, for callers that cannot allocate device
 * memory: code running while a stream is being captured into a CUDA graph (an allocation there
 * fails or breaks the capture), under a memory pool or allocator owned by another framework,
 * or in a process whose device-memory budget is fixed up front.  The paper has no counterpart.
 * Instead of a caller workspace it uses one workspace array compiled into the library's device
 * image (GIRIH_MLP_STATIC_MAX_ROWS rows, about 4.2 MB), which every device that loads the
 * library holds until the process exits.  It calls no cudaMalloc or cudaFree.
 *  - n must be 1..GIRIH_MLP_STATIC_MAX_ROWS; more rows return EINVAL with nothing enqueued.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current and caches it; make that first call before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents; each call writes every
 *    entry it reads, so nothing needs clearing.  Calls whose kernels overlap on the GPU (different
 *    streams, or different host threads) race on the array: order them on one stream.
 * Other arguments and results as girih_mlp_backward.                                         */
#define GIRIH_MLP_STATIC_MAX_ROWS 4096
GIRIH_API int girih_mlp_backward_static(const float* params, const float* X, const float* t, int32_t n, int32_t d,
                                        float* grad, float* loss, void* stream);

/* Optimiser steps on device arrays of np floats. step counts from 1 (Adam bias correction).  */
GIRIH_API int girih_mlp_sgd(float* params, const float* grad, int64_t np, float lr, void* stream);
GIRIH_API int girih_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t np, int64_t step, float lr,
                   float beta1, float beta2, float eps, void* stream);

/* Learned tuning: score the candidates (the given list, or all of girih_tune_candidates when
 * cands is NULL) with the network (device parameters `params`, trained on per-problem centred
 * log GLUP/s), measure the best `k` with girih_tune_measure, set the plan's configuration to the
 * fastest of those and return it in *best.                                                    */
GIRIH_API int girih_tune_learned(girih_plan_t plan, const float* params, const girih_config* cands, int32_t n_cands,
                                 int32_t k, double tol, int64_t max_steps, girih_tune_row* best, int32_t* n_measured);

#ifdef __cplusplus
}
#endif
#endif /* GIRIH_H */
