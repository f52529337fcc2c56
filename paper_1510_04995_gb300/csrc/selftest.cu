// Failure-path check of the blocked kernels' bounded waits: one block runs the RELAXED hand-off
// wait of mwd_kernel.cuh (wait_counts) on progress counters that nothing advances, with a short
// limit.  The wait must give up, set GIRIH_ETIMEOUT in the plan's error word and let the kernel
// return, leaving the context usable.  No GPU fault, trap or endless loop is involved.
#include "mwd_kernel.cuh"
#include "plan.h"

namespace girih {

__global__ void bounded_wait_probe(uint64_t limit_ns, int* err) {
  __shared__ int prog[2];
  if (threadIdx.x == 0) prog[0] = prog[1] = 0;
  __syncthreads();
  if (threadIdx.x == 0) wait_counts(prog, true, true, 1u, limit_ns, err);  // nothing sets prog
  __syncthreads();
}

}  // namespace girih

using namespace girih;

extern "C" {

int girih_check_bounded_wait(girih_plan_t plan, int64_t limit_ns, void* stream) {
  if (!plan) return fail(GIRIH_EINVAL, "plan is NULL");
  if (limit_ns < 1000 || limit_ns > 2000000000LL) return fail(GIRIH_EINVAL, "limit_ns=%lld outside [1e3, 2e9]",
                                                              (long long)limit_ns);
  cudaError_t e = cudaSetDevice(plan->device);
  if (e != cudaSuccess) return cuda_fail(e, "set device");
  bounded_wait_probe<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((uint64_t)limit_ns, plan->err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait probe launch");
  return GIRIH_OK;
}

}  // extern "C"
