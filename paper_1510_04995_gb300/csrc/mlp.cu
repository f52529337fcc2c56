// The learned tuner's network: a 3-layer perceptron D -> 64 -> 64 -> 1 with ReLU, FP32, trained
// on mean squared error.  (The paper's tuner, Sect. 4.2.2, is a measured search; the network is
// an added component that ranks candidate configurations so that only the top few are measured.)
//
// Kernels:
//   mlp_rows         one block handles 4 rows at a time, 64 threads per row (one per hidden unit):
//                    forward pass, and for training the per-row back-propagated signals
//                    (dL/dZ2, dL/dZ1, dL/dy), which are kept in a workspace.
//   mlp_reduce       weight and bias gradients as sums over the rows, one block per output row of
//                    a weight matrix, summed in a fixed order (deterministic), plus the loss.
//   mlp_sgd/adam     element-wise optimiser steps.
// Parameter layout: [W1 (64 x D), b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1)].
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "internal.h"
#include "plan.h"

namespace girih {

constexpr int HID = GIRIH_MLP_HIDDEN;
constexpr int RPB = 4;  // rows per block iteration
constexpr int WS_ROW = 4 * HID + 4;  // workspace floats per row: H1, H2, dZ1, dZ2, dy, err^2

__global__ void __launch_bounds__(HID* RPB) mlp_rows(const float* __restrict__ P, const float* __restrict__ X,
                                                     const float* __restrict__ t, int n, int d,
                                                     float* __restrict__ y, float* __restrict__ ws, int backward) {
  extern __shared__ float sh[];
  float* W1 = sh;                 // 64*d
  float* b1 = W1 + HID * d;       // 64
  float* W2 = b1 + HID;           // 64*64
  float* b2 = W2 + HID * HID;     // 64
  float* W3 = b2 + HID;           // 64
  float* b3 = W3 + HID;           // 1 (+pad)
  float* xs = b3 + 4;             // RPB*d
  float* h1 = xs + RPB * d;       // RPB*64
  float* h2 = h1 + RPB * HID;     // RPB*64
  float* dz2 = h2 + RPB * HID;    // RPB*64
  float* red = dz2 + RPB * HID;   // RPB*64 (reduction scratch)
  const int np = HID * d + HID + HID * HID + HID + HID + 1;
  const int tid = threadIdx.y * HID + threadIdx.x;
  for (int i = tid; i < np; i += HID * RPB) sh[i] = P[i];  // W1..b3 are contiguous in P and sh
  __syncthreads();
  const int j = threadIdx.x, r = threadIdx.y;
  for (int base = blockIdx.x * RPB; base < n; base += gridDim.x * RPB) {
    const int row = base + r;
    const bool ok = row < n;
    for (int i = j; i < d; i += HID) xs[r * d + i] = ok ? X[(size_t)row * d + i] : 0.f;
    __syncthreads();
    float z1 = b1[j];
    for (int i = 0; i < d; ++i) z1 = fmaf(W1[j * d + i], xs[r * d + i], z1);
    const float a1 = fmaxf(z1, 0.f);
    h1[r * HID + j] = a1;
    __syncthreads();
    float z2 = b2[j];
    for (int k = 0; k < HID; ++k) z2 = fmaf(W2[j * HID + k], h1[r * HID + k], z2);
    const float a2 = fmaxf(z2, 0.f);
    h2[r * HID + j] = a2;
    red[r * HID + j] = W3[j] * a2;
    __syncthreads();
    for (int s = HID / 2; s > 0; s >>= 1) {  // tree sum of W3 . h2 over the 64 units of this row
      if (j < s) red[r * HID + j] += red[r * HID + j + s];
      __syncthreads();
    }
    const float yv = red[r * HID] + b3[0];
    if (ok && j == 0 && y) y[row] = yv;
    if (backward) {
      const float e = ok ? yv - t[row] : 0.f;
      const float dy = 2.f * e / (float)n;
      const float g2 = (z2 > 0.f) ? dy * W3[j] : 0.f;
      dz2[r * HID + j] = g2;
      __syncthreads();
      float g1 = 0.f;
      for (int jj = 0; jj < HID; ++jj) g1 = fmaf(dz2[r * HID + jj], W2[jj * HID + j], g1);
      g1 = (z1 > 0.f) ? g1 : 0.f;
      if (ok) {
        float* w = ws + (size_t)row * WS_ROW;
        w[j] = a1;
        w[HID + j] = a2;
        w[2 * HID + j] = g1;
        w[3 * HID + j] = g2;
        if (j == 0) {
          w[4 * HID] = dy;
          w[4 * HID + 1] = e * e;
        }
      }
    }
    __syncthreads();
  }
}

// blockIdx.x in [0, 64): W1 row + b1; [64, 128): W2 row + b2; 128: W3 + b3 + loss.
__global__ void mlp_reduce(const float* __restrict__ X, int n, int d, const float* __restrict__ ws,
                           float* __restrict__ grad, float* __restrict__ loss) {
  const int g = blockIdx.x, c = threadIdx.x;
  float* gW1 = grad;
  float* gb1 = gW1 + HID * d;
  float* gW2 = gb1 + HID;
  float* gb2 = gW2 + HID * HID;
  float* gW3 = gb2 + HID;
  float* gb3 = gW3 + HID;
  if (g < HID) {
    const int jr = g;
    if (c < d) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s = fmaf(ws[(size_t)i * WS_ROW + 2 * HID + jr], X[(size_t)i * d + c], s);
      gW1[jr * d + c] = s;
    } else if (c == d) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s += ws[(size_t)i * WS_ROW + 2 * HID + jr];
      gb1[jr] = s;
    }
  } else if (g < 2 * HID) {
    const int jr = g - HID;
    if (c < HID) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s = fmaf(ws[(size_t)i * WS_ROW + 3 * HID + jr], ws[(size_t)i * WS_ROW + c], s);
      gW2[jr * HID + c] = s;
    } else if (c == HID) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s += ws[(size_t)i * WS_ROW + 3 * HID + jr];
      gb2[jr] = s;
    }
  } else {
    if (c < HID) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s = fmaf(ws[(size_t)i * WS_ROW + 4 * HID], ws[(size_t)i * WS_ROW + HID + c], s);
      gW3[c] = s;
    } else if (c == HID) {
      float s = 0.f;
      for (int i = 0; i < n; ++i) s += ws[(size_t)i * WS_ROW + 4 * HID];
      gb3[0] = s;
    } else if (c == HID + 1 && loss) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += ws[(size_t)i * WS_ROW + 4 * HID + 1];
      loss[0] = (float)(s / n);
    }
  }
}

__global__ void mlp_sgd_kernel(float* p, const float* g, int64_t np, float lr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
    p[i] -= lr * g[i];
}

__global__ void mlp_adam_kernel(float* p, const float* g, float* m, float* v, int64_t np, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

static size_t rows_smem(int d) {
  return sizeof(float) * ((size_t)HID * d + HID + HID * HID + HID + HID + 4 + RPB * d + 4 * RPB * HID);
}

int mlp_forward_impl(const float* P, const float* X, int n, int d, float* y, float* ws, float* t, float* grad,
                     float* loss, cudaStream_t st) {
  if (n < 1 || d < 1 || d > HID || !P || !X) return fail(GIRIH_EINVAL, "bad network arguments (need 1 <= d <= 64)");
  const size_t sm = rows_smem(d);
  cudaError_t e = cudaFuncSetAttribute(mlp_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return cuda_fail(e, "mlp attributes");
  const int blocks = (n + RPB - 1) / RPB < 304 ? (n + RPB - 1) / RPB : 304;
  const bool bw = grad != nullptr;
  mlp_rows<<<blocks, dim3(HID, RPB), sm, st>>>(P, X, t, n, d, y, ws, bw ? 1 : 0);
  if (bw) mlp_reduce<<<2 * HID + 1, HID + 2, 0, st>>>(X, n, d, ws, grad, loss);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mlp launch");
  return GIRIH_OK;
}

// Workspace of the allocation-free backward pass (girih_mlp_backward_static): a fixed array in
// the library's device image, GIRIH_MLP_STATIC_MAX_ROWS rows of WS_ROW floats (4.2 MB), present
// on every device that loads the library until the process exits.
__device__ __align__(256) float g_mlp_static_ws[(size_t)GIRIH_MLP_STATIC_MAX_ROWS * WS_ROW];

// Device address of g_mlp_static_ws, looked up once per device (with that device current).
static float* static_ws_address(int* rc) {
  static std::mutex mu;
  static float* addr[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    *rc = cuda_fail(e == cudaSuccess ? cudaErrorInvalidDevice : e, "current device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mlp_static_ws);
    if (e != cudaSuccess) {
      *rc = cuda_fail(e, "cudaGetSymbolAddress of the static workspace");
      return nullptr;
    }
    addr[dev] = static_cast<float*>(p);
  }
  *rc = GIRIH_OK;
  return addr[dev];
}

}  // namespace girih

using namespace girih;

extern "C" {

int girih_mlp_backward_static(const float* params, const float* X, const float* t, int32_t n, int32_t d,
                              float* grad, float* loss, void* stream) {
  if (!t || !grad) return fail(GIRIH_EINVAL, "targets and gradient are required");
  if (n < 1 || n > GIRIH_MLP_STATIC_MAX_ROWS)
    return fail(GIRIH_EINVAL, "n=%d rows: the allocation-free backward pass takes 1..%d rows", n,
                GIRIH_MLP_STATIC_MAX_ROWS);
  int rc = GIRIH_OK;
  float* ws = static_ws_address(&rc);
  if (!ws) return rc;
  // every workspace entry the gradient sums read is written by this call first (no clearing needed)
  return mlp_forward_impl(params, X, n, d, nullptr, ws, const_cast<float*>(t), grad, loss,
                          static_cast<cudaStream_t>(stream));
}

int64_t girih_mlp_num_params(int32_t d) { return (int64_t)HID * d + HID + HID * HID + HID + HID + 1; }

int64_t girih_mlp_workspace_floats(int32_t n) { return (int64_t)n * WS_ROW + 64; }

int girih_mlp_forward(const float* params, const float* X, int32_t n, int32_t d, float* y, float* workspace,
                      void* stream) {
  if (!y) return fail(GIRIH_EINVAL, "y is NULL");
  return mlp_forward_impl(params, X, n, d, y, workspace, nullptr, nullptr, nullptr,
                          static_cast<cudaStream_t>(stream));
}

int girih_mlp_backward(const float* params, const float* X, const float* t, int32_t n, int32_t d, float* grad,
                       float* loss, float* workspace, void* stream) {
  if (!t || !grad || !workspace) return fail(GIRIH_EINVAL, "targets, gradient and workspace are required");
  return mlp_forward_impl(params, X, n, d, nullptr, workspace, const_cast<float*>(t), grad, loss,
                          static_cast<cudaStream_t>(stream));
}

int girih_mlp_sgd(float* params, const float* grad, int64_t np, float lr, void* stream) {
  if (!params || !grad || np < 1) return fail(GIRIH_EINVAL, "bad sgd arguments");
  const int blocks = (int)((np + 255) / 256 < 1024 ? (np + 255) / 256 : 1024);
  mlp_sgd_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, np, lr);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GIRIH_OK : cuda_fail(e, "sgd launch");
}

int girih_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t np, int64_t step, float lr,
                   float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || np < 1 || step < 1) return fail(GIRIH_EINVAL, "bad adam arguments");
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  const int blocks = (int)((np + 255) / 256 < 1024 ? (np + 255) / 256 : 1024);
  mlp_adam_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, np, lr, beta1, beta2,
                                                                         eps, c1, c2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GIRIH_OK : cuda_fail(e, "adam launch");
}

}  // extern "C"
