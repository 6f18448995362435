// Small kernels of the step: squared-L2 loss and dL/dE (row a8), max |dL/dE|
// for the deterministic adjoint, fixed point -> float, and Adam (row a10).
#include <algorithm>

#include "fr_internal.h"

namespace fr {
namespace {

// L = sum over interior pixels of (E - E_ref)^2; dL/dE = 2 (E - E_ref) there and
// 0 on ghost pixels. A fixed grid of kLossBlocks blocks writes one partial sum
// each; the last block to finish adds them with a fixed-shape tree (the result
// is bit-identical from run to run) and re-arms the counter for the next launch.
__device__ __forceinline__ double block_sum(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? s_red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ E, const float* __restrict__ Eref, int nx,
                                              int ny, int hx, int hy, int ncol, int nrow,
                                              double* __restrict__ partials, unsigned int* counter,
                                              double* __restrict__ loss, float* __restrict__ dLdE) {
  double acc = 0.0;
  const int n = ncol * nrow;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int r = q / ncol, c = q - r * ncol;
    const int i = c - hx, j = r - hy;
    float g = 0.0f;
    if (i >= 0 && i < nx && j >= 0 && j < ny) {
      const float d = E[q] - Eref[j * nx + i];
      acc += (double)d * (double)d;
      g = 2.0f * d;
    }
    dLdE[q] = g;
  }
  __shared__ double s_red[8];
  __shared__ bool s_last;
  const double b = block_sum(acc, s_red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double v = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) v += __ldcg(partials + q);
    __syncthreads();
    const double total = block_sum(v, s_red);
    if (threadIdx.x == 0) {
      *loss = total;
      *counter = 0u;
    }
  }
}

// max |x| into *out (out must start at 0); non-negative floats order like their bits.
__global__ void k_absmax(const float* __restrict__ x, size_t n, float* out) {
  float m = 0.0f;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[q]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(m));
}

__global__ void k_fix_to_float(const unsigned long long* __restrict__ q, float* __restrict__ out, size_t n,
                               float inv_scale, int accumulate) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = (float)((double)(long long)q[i] * (double)inv_scale);
  out[i] = accumulate ? out[i] + v : v;
}

// Adam (Kingma & Ba, Algorithm 1) in one block, so that every thread reads the
// same step count before thread 0 advances it.
__global__ void __launch_bounds__(1024) k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                                               const float* __restrict__ g, int64_t n, float lr, float b1, float b2,
                                               float eps, int32_t* step) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = *step + 1;
  __syncthreads();
  const int t = s_t;
  const float bc1 = 1.0f - powf(b1, (float)t);
  const float bc2 = 1.0f - powf(b2, (float)t);
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    const float gq = g[q];
    const float mq = fmaf(b1, m[q], (1.0f - b1) * gq);
    const float vq = fmaf(b2, v[q], (1.0f - b2) * gq * gq);
    m[q] = mq;
    v[q] = vq;
    P[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
  }
  if (threadIdx.x == 0) *step = t;
}

}  // namespace

cudaError_t launch_loss(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y, double* partials,
                        unsigned int* counter, double* loss, float* dLdE, cudaStream_t st) {
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  k_loss<<<kLossBlocks, 256, 0, st>>>(E, Eref, nx, ny, (nu_x - 1) / 2, (nu_y - 1) / 2, ncol, nrow, partials,
                                      counter, loss, dLdE);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const float* x, size_t n, float* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<size_t>(120, (n + 255) / 256);
  k_absmax<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fix_to_float(const unsigned long long* q, float* out, size_t n, float inv_scale, int accumulate,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_fix_to_float<<<(unsigned int)((n + 255) / 256), 256, 0, st>>>(q, out, n, inv_scale, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* P, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2,
                        float eps, int32_t* step, cudaStream_t st) {
  k_adam<<<1, 1024, 0, st>>>(P, m, v, g, n, lr, b1, b2, eps, step);
  return cudaGetLastError();
}

}  // namespace fr
