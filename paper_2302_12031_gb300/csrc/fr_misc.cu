// Small kernels of the step: max |dL/dE| for the deterministic adjoint, fixed
// point -> float, and Adam (row a10).
#include <algorithm>

#include "fr_device.cuh"

namespace fr {
namespace {

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
  pdl_wait();      // the gradient is the previous kernel's output
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

// Zeroes the buffers of a ZeroList: 16-byte stores where a buffer is aligned,
// bytes at its unaligned ends. Lets the next kernel (a forward launched early)
// begin at once; it waits for this one before it writes.
__global__ void __launch_bounds__(256) k_zero_list(const __grid_constant__ ZeroList z) {
  pdl_trigger();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < z.n; ++k) {
    unsigned char* p = static_cast<unsigned char*>(z.ptr[k]);
    const uint64_t n = z.bytes[k];
    const uint64_t lead = (uint64_t)((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15);
    const uint64_t head = lead < n ? lead : n;
    const uint64_t nv = (n - head) / 16;
    uint4* pv = reinterpret_cast<uint4*>(p + head);
    for (uint64_t i = t0; i < nv; i += stride) pv[i] = make_uint4(0u, 0u, 0u, 0u);
    const uint64_t tail0 = head + nv * 16;
    for (uint64_t i = t0; i < head; i += stride) p[i] = 0;
    for (uint64_t i = tail0 + t0; i < n; i += stride) p[i] = 0;
  }
}

}  // namespace

cudaError_t launch_zero_list(const ZeroList& z, cudaStream_t st) {
  uint64_t most = 0;
  for (int k = 0; k < z.n; ++k) most = std::max<uint64_t>(most, z.bytes[k]);
  if (most == 0) return cudaSuccess;
  const uint64_t blocks = std::min<uint64_t>(152, (most / 16 + 255) / 256 + 1);
  k_zero_list<<<(unsigned int)blocks, 256, 0, st>>>(z);
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
                        float eps, int32_t* step, cudaStream_t st, bool pdl) {
  return launch_k(k_adam, dim3(1), dim3(1024), 0, st, pdl, P, m, v, g, n, lr, b1, b2, eps, step);
}

}  // namespace fr
