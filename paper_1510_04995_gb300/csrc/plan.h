// The opaque plan behind girih_plan_t, and helpers shared by api.cu and tuner.cu.
#pragma once
#include <cstdarg>
#include <cstdint>

#include "internal.h"

struct girih_plan_s {
  int32_t stencil = 0, dtype = 0, R = 1, elem = 8;
  int64_t nx = 0, ny = 0, nz = 0, ldx = 0, T = 0, gstride = 0;
  int device = 0, sm_count = 0;
  int64_t smem_optin = 0;
  girih_config cfg{};
  // device buffers owned by the plan: girih_run_host staging and the tuner's own arrays
  void* host_u = nullptr;
  void* host_up = nullptr;
  void* host_co = nullptr;
  void* tune_u = nullptr;
  void* tune_up = nullptr;
  void* tune_co = nullptr;
  int* err = nullptr;  // device error word of the kernels' bounded waits
  // persistent schedule: item list + per-row table, completion flags, FIFO counter, run epoch
  int* sched = nullptr;
  int64_t sched_cap = 0;  // ints
  int64_t sched_T = -1;   // diamond rows, width and z segment of the uploaded list
  int32_t sched_dw = 0, sched_zs = 0;
  int* flags = nullptr;
  int64_t flags_cap = 0;  // ints
  int* fifo = nullptr;
  int32_t epoch = 0;
  bool bulk_layout = false;  // rows are 16-byte multiples: the blocked kernel may use bulk copies
};

namespace girih {
using Plan = girih_plan_s;
int fail(int code, const char* fmt, ...);
void g_err_clear();
int cuda_fail(cudaError_t e, const char* where);
// Validates a configuration for the plan's device and layout.  ptrs16: the buffers of the run
// are 16-byte aligned (plan-time checks assume so); mv_out: the kernel's data path.
int check_config(const Plan* p, const girih_config* c, int64_t* smem_out, int* xw_out, int* g_out,
                 int* mv_out = nullptr, bool ptrs16 = true, int* lead_out = nullptr);
int run_sweep(Plan* p, int64_t T, void* u, void* u_prev, const void* coeffs, const double* c,
              const girih_config& cfg, cudaStream_t st);
int64_t mwd_rows(int64_t T, int dw, int R);
// x slab per block of the blocked kernel for a cluster of C blocks on data path mv
int slab_width(const Plan* p, int C, int mv);
}  // namespace girih
