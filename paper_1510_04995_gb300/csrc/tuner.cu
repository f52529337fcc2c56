// Auto-tuner (arXiv 1510.04995, Sect. 4.2.2) and the learned tuner built on it.
//
// Exhaustive tuning: every configuration of the search space (naive sweep; for the blocked
// sweep every diamond width D_w, wavefront width N_F, cluster size -- the thread-group size of
// the paper -- and block size) is pruned by feasibility (the tile's shared-memory footprint, the
// GPU counterpart of the cache-block-size model of Eq. 3, against the per-block limit; cluster
// schedulability), then measured on tuner-owned arrays (Sect. 4.2.2: the tuner allocates and
// initialises its own arrays).  The test length grows in whole diamond rows until two
// consecutive measurements agree within a relative threshold, and the longest test is reported.
//
// Learned tuning: the network of mlp.cu scores every feasible candidate from its features; only
// the k best-scored are measured, the fastest of those is chosen.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace girih {

int mlp_forward_impl(const float* P, const float* X, int n, int d, float* y, float* ws, float* t, float* grad,
                     float* loss, cudaStream_t st);

// Deterministic fill of the tuner's arrays: u = u_prev (so halos agree) with values in [-1, 1),
// coefficients set to constants that keep the first-order stencils' weights summing to one.
template <typename T>
__global__ void tune_fill(T* u, T* up, T* co, int64_t n, int ncoef) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    const T v = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    u[i] = v;
    up[i] = v;
    for (int g = 0; g < ncoef; ++g) co[g * n + i] = (ncoef == 7) ? (T)(1.0 / 7.0) : (ncoef == 1 ? (T)0.75 : (T)0.003);
  }
}

static int ensure_tune_arrays(Plan* p) {
  const int nc = ncoef_of(p->stencil);
  const size_t bytes = (size_t)(p->gstride * p->elem);
  cudaError_t e = cudaSuccess;
  if (!p->tune_u) e = cudaMalloc(&p->tune_u, bytes);
  if (e == cudaSuccess && !p->tune_up) e = cudaMalloc(&p->tune_up, bytes);
  if (e == cudaSuccess && nc > 0 && !p->tune_co) e = cudaMalloc(&p->tune_co, bytes * nc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GIRIH_ENOMEM, "tuner arrays: %s", cudaGetErrorString(e));
  }
  return GIRIH_OK;
}

static cudaError_t fill(Plan* p, cudaStream_t st) {
  const int nc = ncoef_of(p->stencil);
  const int blocks = 152 * 8;
  if (p->dtype == GIRIH_F64)
    tune_fill<double><<<blocks, 256, 0, st>>>((double*)p->tune_u, (double*)p->tune_up, (double*)p->tune_co,
                                             p->gstride, nc);
  else
    tune_fill<float><<<blocks, 256, 0, st>>>((float*)p->tune_u, (float*)p->tune_up, (float*)p->tune_co, p->gstride,
                                            nc);
  return cudaGetLastError();
}

static const double kC7[5] = {0.4, 0.1, 0, 0, 0};
static const double kC25[5] = {-0.9, 0.05, 0.025, 0.0125, 0.00625};
static const double kCBox[5] = {0.4, 0.05, 0.02, 0.0075, 0};
static const double kCRB[5] = {0.0, 1.0 / 6.0, 0, 0, 0};

int measure(Plan* p, const girih_config& cfg, double tol, int64_t max_steps, girih_tune_row* row) {
  const auto wall0 = std::chrono::steady_clock::now();
  int rc = check_config(p, &cfg, &row->smem, nullptr, nullptr);
  if (rc != GIRIH_OK) return rc;
  rc = ensure_tune_arrays(p);
  if (rc != GIRIH_OK) return rc;
  const double* c = is_box(p->stencil) ? kCBox : (p->stencil == GIRIH_7PT_RBGS ? kCRB : (p->R == 4 ? kC25 : kC7));
  // one diamond row advances H/2 steps; grow the test in units of two rows (Sect. 4.2.2)
  const int64_t unit = (cfg.algo == GIRIH_ALGO_MWD) ? std::max<int64_t>(cfg.dw / p->R, 2) : 2;
  int64_t steps = unit;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const cudaStream_t st = 0;
  double prev = -1.0, glups = 0.0, secs = 0.0;
  int64_t used = steps;
  cudaError_t ce = fill(p, st);
  // warm-up run (module load, attributes)
  if (ce == cudaSuccess) rc = run_sweep(p, unit, p->tune_u, p->tune_up, p->tune_co, c, cfg, st);
  while (rc == GIRIH_OK && ce == cudaSuccess) {
    ce = fill(p, st);
    if (ce != cudaSuccess) break;
    cudaEventRecord(e0, st);
    rc = run_sweep(p, steps, p->tune_u, p->tune_up, p->tune_co, c, cfg, st);
    cudaEventRecord(e1, st);
    ce = cudaEventSynchronize(e1);
    if (rc != GIRIH_OK || ce != cudaSuccess) break;
    rc = girih_status(p, nullptr);
    if (rc != GIRIH_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    secs = ms * 1e-3;
    glups = (double)p->nx * p->ny * p->nz * steps / secs * 1e-9;
    used = steps;
    if (prev > 0 && std::fabs(glups - prev) <= tol * glups) break;
    if (steps * 2 > max_steps) break;
    prev = glups;
    steps *= 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ce, "tuner measurement");
  if (rc != GIRIH_OK) return rc;
  row->cfg = cfg;
  row->glups = glups;
  row->seconds = secs;
  row->steps = used;
  row->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
  return GIRIH_OK;
}

std::vector<girih_config> candidates(Plan* p) {
  std::vector<girih_config> out;
  out.push_back(girih_config{GIRIH_ALGO_NAIVE, 0, 1, 1, 256, GIRIH_FED});
  const int R = p->R;
  for (int dw = 2 * R; dw <= 64 * R; dw += 2 * R)
    for (int nf : {1, 2})
      for (int C : {1, 2, 4, 8, 16})
        for (int th : {128, 256, 512, 1024})
          for (int v : {GIRIH_FED, GIRIH_RELAXED, GIRIH_FED_BULK, GIRIH_FED_ELEM, GIRIH_RELAXED_ELEM,
                        GIRIH_FED_PERSISTENT}) {
            if ((v == GIRIH_RELAXED || v == GIRIH_RELAXED_ELEM) && C == 1) continue;  // one block: = FED
            // on an unaligned layout FED is already the element path
            if ((v == GIRIH_FED_ELEM || v == GIRIH_RELAXED_ELEM) && !p->bulk_layout) continue;
            girih_config c{GIRIH_ALGO_MWD, dw, nf, C, th, v};
            if (check_config(p, &c, nullptr, nullptr, nullptr) == GIRIH_OK) out.push_back(c);
          }
  // RELAXED_PERSISTENT: blocks sized to the tile's tasks (1, 2 or 4 per computing thread, whole
  // warps) plus the two data-moving warps
  if (async_stencil(p->stencil) && p->bulk_layout)
    for (int dw = 2 * R; dw <= 64 * R; dw += 2 * R)
      for (int C : {1, 2, 4, 8, 16}) {
        const int64_t tasks = (int64_t)mwd_max_pairs(R, dw) * (slab_width(p, C, MV_ASYNC) / mwd_vx(p->stencil,
                                                                                                   p->dtype, MV_ASYNC));
        int last = 0;
        for (int G : {1, 2, 4}) {
          const int th = (int)std::max<int64_t>(32, (tasks + 32LL * G - 1) / (32LL * G) * 32) + kAsyncMovers;
          if (th == last || th > async_max_threads(G, ncoef_of(p->stencil) > 0)) continue;
          last = th;
          girih_config c{GIRIH_ALGO_MWD, dw, 1, C, th, GIRIH_RELAXED_PERSISTENT};
          if (check_config(p, &c, nullptr, nullptr, nullptr) == GIRIH_OK) out.push_back(c);
        }
      }
  // OVERLAP_PERSISTENT: blocks sized to the tasks of the widened levels the same way
  if (ovl_stencil(p->stencil) && p->bulk_layout)
    for (int dw = 2 * R; dw <= 64 * R; dw += 2 * R)
      for (int C : {1, 2, 4, 8, 16}) {
        const int64_t tasks =
            mwd_ovl_tasks(R, dw, slab_width(p, C, MV_OVL), mwd_vx(p->stencil, p->dtype, MV_OVL), 16 / p->elem);
        int last = 0;
        for (int G : {1, 2, 4}) {
          const int th = (int)std::max<int64_t>(32, (tasks + 32LL * G - 1) / (32LL * G) * 32) + kOvlMovers;
          if (th == last || th > async_max_threads(G, ncoef_of(p->stencil) > 0, R == 4)) continue;
          last = th;
          girih_config c{GIRIH_ALGO_MWD, dw, 1, C, th, GIRIH_OVERLAP_PERSISTENT};
          if (check_config(p, &c, nullptr, nullptr, nullptr) != GIRIH_OK) continue;
          out.push_back(c);
          // rows of fewer diamonds than the device has clusters: also split the tiles along z
          // (Sect. 8), so that the next row's diamonds start before this row's finish
          if ((p->ny + dw - 1) / dw + 1 < std::max(p->sm_count / C, 1))
            for (int zs : {32, 64, 128}) {
              if (zs >= p->nz) break;
              c.zseg = zs;
              if (check_config(p, &c, nullptr, nullptr, nullptr) == GIRIH_OK) out.push_back(c);
            }
        }
      }
  g_err_clear();
  return out;
}

}  // namespace girih

using namespace girih;

extern "C" {

int girih_tune_candidates(girih_plan_t plan, girih_config* out, int32_t cap, int32_t* count) {
  if (!plan || !count) return fail(GIRIH_EINVAL, "NULL argument");
  const std::vector<girih_config> c = candidates(plan);
  const int n = (int)c.size();
  for (int i = 0; i < n && i < cap && out; ++i) out[i] = c[i];
  *count = n;
  return GIRIH_OK;
}

int girih_tune_measure(girih_plan_t plan, const girih_config* cfg, double tol, int64_t max_steps,
                       girih_tune_row* row) {
  if (!plan || !cfg || !row) return fail(GIRIH_EINVAL, "NULL argument");
  if (tol <= 0 || max_steps < 1) return fail(GIRIH_EINVAL, "tol must be > 0 and max_steps >= 1");
  return measure(plan, *cfg, tol, max_steps, row);
}

static void append_csv(FILE* f, const Plan* p, const girih_tune_row& r) {
  fprintf(f, "%d,%d,%lld,%lld,%lld,%d,%d,%d,%d,%d,%d,%.6f,%.6e,%lld,%lld,%.6e,%d\n", p->stencil, p->dtype,
          (long long)p->nx, (long long)p->ny, (long long)p->nz, r.cfg.algo, r.cfg.dw, r.cfg.nf, r.cfg.cluster,
          r.cfg.threads, r.cfg.variant, r.glups, r.seconds, (long long)r.steps, (long long)r.smem, r.tune_seconds,
          r.cfg.zseg);
}

static int candidate_list(Plan* p, const girih_config* given, int32_t n, std::vector<girih_config>* out) {
  if (!given) {
    *out = candidates(p);
    return GIRIH_OK;
  }
  if (n < 1) return fail(GIRIH_EINVAL, "empty candidate list");
  out->assign(given, given + n);
  for (const girih_config& c : *out) {
    const int rc = check_config(p, &c, nullptr, nullptr, nullptr);
    if (rc != GIRIH_OK) return rc;
  }
  return GIRIH_OK;
}

int girih_tune_exhaustive(girih_plan_t plan, const girih_config* cand_list, int32_t n_cands, double tol,
                          int64_t max_steps, const char* db_path, girih_tune_row* best, int32_t* n_measured) {
  if (!plan || !best) return fail(GIRIH_EINVAL, "NULL argument");
  std::vector<girih_config> cands;
  const int crc = candidate_list(plan, cand_list, n_cands, &cands);
  if (crc != GIRIH_OK) return crc;
  FILE* f = nullptr;
  if (db_path) {
    f = fopen(db_path, "a");
    if (!f) return fail(GIRIH_EINVAL, "cannot open %s", db_path);
  }
  girih_tune_row top{};
  top.glups = -1;
  int nm = 0;
  for (const girih_config& c : cands) {
    girih_tune_row r{};
    const int rc = measure(plan, c, tol, max_steps, &r);
    if (rc != GIRIH_OK) {
      if (f) fclose(f);
      return rc;
    }
    ++nm;
    if (f) append_csv(f, plan, r);
    if (r.glups > top.glups) top = r;
  }
  if (f) fclose(f);
  plan->cfg = top.cfg;
  *best = top;
  if (n_measured) *n_measured = nm;
  return GIRIH_OK;
}

int girih_mlp_features(int32_t stencil, int32_t dtype, int64_t nx, int64_t ny, int64_t nz, const girih_config* cfg,
                       float* out) {
  if (!cfg || !out || stencil < 0 || stencil > 6) return fail(GIRIH_EINVAL, "bad feature arguments");
  for (int i = 0; i < GIRIH_MLP_FEATURES; ++i) out[i] = 0.f;
  out[stencil == GIRIH_25PT_CGRID ? GIRIH_25PT_CONST : (stencil >= GIRIH_27PT_BOX ? GIRIH_7PT_CONST : stencil)] = 1.f;
  out[4] = dtype == GIRIH_F32 ? 1.f : 0.f;
  out[5] = (float)(std::log2((double)nx) / 10.0);
  out[6] = (float)(std::log2((double)ny) / 10.0);
  out[7] = (float)(std::log2((double)nz) / 10.0);
  const bool mwd = cfg->algo == GIRIH_ALGO_MWD;
  out[8] = mwd ? 1.f : 0.f;
  const int R = radius_of(stencil);
  out[9] = mwd ? (float)cfg->dw / (16.f * R) : 0.f;
  out[10] = mwd ? (float)cfg->nf / 2.f : 0.f;
  out[11] = mwd ? (float)std::log2((double)cfg->cluster) / 4.f : 0.f;
  out[12] = (float)cfg->threads / 512.f;
  out[13] = (float)cfg->variant;
  const int nd = 2 + ncoef_of(stencil);
  const int elem = dtype == GIRIH_F64 ? 8 : 4;
  const double bc = mwd ? girih_model_code_balance(cfg->dw, R, nd, elem) : (double)(nd + 1 - (second_order(stencil) ? 0 : 1)) * elem;
  out[14] = (float)(std::log2(std::max(bc, 0.25)) / 8.0);
  // x slab per block relative to a warp: wide slabs amortise the x halo
  int64_t w = mwd ? (nx + cfg->cluster - 1) / cfg->cluster : nx;
  out[15] = (float)(std::log2((double)std::max<int64_t>(w, 1)) / 10.0);
  return GIRIH_OK;
}

int girih_tune_learned(girih_plan_t plan, const float* params, const girih_config* cand_list, int32_t n_cands,
                       int32_t k, double tol, int64_t max_steps, girih_tune_row* best, int32_t* n_measured) {
  if (!plan || !params || !best || k < 1) return fail(GIRIH_EINVAL, "bad arguments");
  std::vector<girih_config> cands;
  const int crc = candidate_list(plan, cand_list, n_cands, &cands);
  if (crc != GIRIH_OK) return crc;
  const int n = (int)cands.size(), d = GIRIH_MLP_FEATURES;
  std::vector<float> X((size_t)n * d), y(n);
  for (int i = 0; i < n; ++i)
    girih_mlp_features(plan->stencil, plan->dtype, plan->nx, plan->ny, plan->nz, &cands[i], &X[(size_t)i * d]);
  float *dX = nullptr, *dy = nullptr;
  cudaError_t e = cudaMalloc(&dX, X.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dy, y.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice);
  int rc = GIRIH_OK;
  if (e == cudaSuccess) rc = mlp_forward_impl(params, dX, n, d, dy, nullptr, nullptr, nullptr, nullptr, 0);
  if (e == cudaSuccess && rc == GIRIH_OK) e = cudaMemcpy(y.data(), dy, y.size() * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(dX);
  cudaFree(dy);
  if (e != cudaSuccess) return cuda_fail(e, "learned tuner scoring");
  if (rc != GIRIH_OK) return rc;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] > y[b]; });
  girih_tune_row top{};
  top.glups = -1;
  int nm = 0;
  for (int i = 0; i < n && nm < k; ++i) {
    girih_tune_row r{};
    rc = measure(plan, cands[order[i]], tol, max_steps, &r);
    if (rc != GIRIH_OK) return rc;
    ++nm;
    if (r.glups > top.glups) top = r;
  }
  plan->cfg = top.cfg;
  *best = top;
  if (n_measured) *n_measured = nm;
  return GIRIH_OK;
}

}  // extern "C"
