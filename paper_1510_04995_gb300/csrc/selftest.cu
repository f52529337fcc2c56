// Device self-checks and measurements that are not part of the paper's method:
//  * the failure-path check of the blocked kernels' bounded waits: one block runs the RELAXED
//    hand-off wait of mwd_kernel.cuh (wait_counts) on progress counters that nothing advances,
//    with a short limit.  The wait must give up, set GIRIH_ETIMEOUT in the plan's error word and
//    let the kernel return, leaving the context usable.  No GPU fault, trap or endless loop.
//  * the fused multiply-add rate of the GPU in FP64 and FP32, the denominator of the FP64
//    sweeps' arithmetic roofline (every SM runs independent FMA chains for about 0.1 s).
#include <chrono>

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

// Eight independent FMA chains per thread; the result is stored only if it takes a value it
// cannot take, so the chains stay live without a memory stream.
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = Ops<T>::fma(x[j], a, b);
  }
  T s = x[0];
#pragma unroll
  for (int j = 1; j < 8; ++j) s = Ops<T>::add(s, x[j]);
  if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int fma_rate(int sms, double* rate, double* secs, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel<T>, 256, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  const int blocks = sms * per_sm;
  T* sink = nullptr;
  e = cudaMalloc(&sink, (size_t)blocks * 256 * sizeof(T));
  if (e != cudaSuccess) return fail(GIRIH_ENOMEM, "sink: %s", cudaGetErrorString(e));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a short calibration run, then one sized to about 0.1 s
  int iters = 1 << 12;
  double sec = 0.0;
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    cudaEventRecord(e0, st);
    fma_rate_kernel<T><<<blocks, 256, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    sec = ms * 1e-3;
    if (pass == 0) iters = (int)std::min<double>(1 << 30, std::max<double>(iters, iters * 0.1 / std::max(sec, 1e-6)));
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "FMA rate kernel");
  *rate = (double)blocks * 256.0 * 8.0 * (double)iters / sec;
  *secs = sec;
  return GIRIH_OK;
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

int girih_measure_fma_rate(int32_t dtype, double* fma_per_s, double* seconds, void* stream) {
  if (!fma_per_s) return fail(GIRIH_EINVAL, "fma_per_s is NULL");
  if (dtype != GIRIH_F64 && dtype != GIRIH_F32) return fail(GIRIH_EINVAL, "unknown dtype %d", dtype);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  double secs = 0.0;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int rc = dtype == GIRIH_F64 ? fma_rate<double>(sms, fma_per_s, &secs, st) : fma_rate<float>(sms, fma_per_s, &secs, st);
  if (rc == GIRIH_OK && seconds) *seconds = secs;
  return rc;
}

}  // extern "C"
