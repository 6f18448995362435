// Throughput probes of the SM resources the trace kernels use: FP32 FMA
// (scalar and packed pairs), the XU pipe (MUFU ex2 and rsqrt, float <-> int
// conversions), shared-memory atomics at random addresses (u32 and f32) and
// 16-byte global float reductions at random L2-resident addresses. They are a
// measurement aid for the roofline of the traces, not part of the method: the
// caller times one launch with CUDA events on its stream and divides the
// operation count fr_probe returns by that time.
#include <cstdint>

#include "fr_internal.h"

namespace fr {
namespace {

constexpr int kChains = 8;                 // independent dependency chains per thread
constexpr int kSharedWords = 16384;        // random-address table in shared memory (64 KB)

__device__ __forceinline__ float ex2_probe(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_probe(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 fma2_probe(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;"
               : "=l"(d)
               : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
                 "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

// KIND: 0 FFMA, 1 packed FFMA2, 2 ex2, 3 rsqrt, 4 float->int->float,
// 5 shared u32 atomics, 6 shared f32 atomics, 7 global float4 reductions.
template <int KIND>
__global__ void __launch_bounds__(1024) k_probe(int iters, float* out, int n_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.0f;
  if constexpr (KIND <= 4) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.5f + 1e-3f * (float)((tid + j) & 255);
    const float m = 0.999f, c = 1e-4f;
    for (int i = 0; i < iters; ++i) {
      if constexpr (KIND == 0) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], m, c);
      } else if constexpr (KIND == 1) {
#pragma unroll
        for (int j = 0; j < kChains; j += 2) {
          const float2 r = fma2_probe(make_float2(a[j], a[j + 1]), make_float2(m, m), make_float2(c, c));
          a[j] = r.x;
          a[j + 1] = r.y;
        }
      } else if constexpr (KIND == 2) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = ex2_probe(-a[j]);
      } else if constexpr (KIND == 3) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = rsqrt_probe(a[j]);
      } else {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = (float)__float2int_rz(a[j] * 3.0f) * 0.25f + 0.5f;
      }
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += a[j];
  } else if constexpr (KIND == 5 || KIND == 6) {
    unsigned int* tab = reinterpret_cast<unsigned int*>(smem);
    for (int q = threadIdx.x; q < kSharedWords; q += blockDim.x) tab[q] = 0u;
    __syncthreads();
    uint32_t x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = 0x9E3779B9u * (uint32_t)(tid * 4 + j + 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = x[j] * 1664525u + 1013904223u;
        const uint32_t k = x[j] >> 18;   // 14 bits: kSharedWords
        if constexpr (KIND == 5) atomicAdd(tab + k, 1u);
        else atomicAdd(reinterpret_cast<float*>(tab) + k, 1.0f);
      }
    }
    __syncthreads();
    acc = (float)tab[threadIdx.x & (kSharedWords - 1)];
  } else {
    uint32_t x[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) x[j] = 0x9E3779B9u * (uint32_t)(tid * 2 + j + 1);
    const uint32_t groups = (uint32_t)(n_out / 4);   // a power of two
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        x[j] = x[j] * 1664525u + 1013904223u;
        const uint32_t g = (x[j] >> 8) & (groups - 1);
        atomicAdd(reinterpret_cast<float4*>(out) + g, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
      }
    }
    return;
  }
  if (tid < n_out) out[tid] = acc;
}

using ProbeKernel = void (*)(int, float*, int);

ProbeKernel probe_kernel(int kind) {
  switch (kind) {
    case 0: return k_probe<0>;
    case 1: return k_probe<1>;
    case 2: return k_probe<2>;
    case 3: return k_probe<3>;
    case 4: return k_probe<4>;
    case 5: return k_probe<5>;
    case 6: return k_probe<6>;
    default: return k_probe<7>;
  }
}

}  // namespace

// Operations one launch performs: FP32 flops (FMA = 2) for kinds 0-1, thread
// operations on the XU pipe for 2-4 (a conversion round trip is two), atomic
// thread operations for 5-6 and 16-byte reductions for 7.
double probe_ops(int kind, int blocks, int threads, int iters) {
  const double t = (double)blocks * threads * iters;
  switch (kind) {
    case 0:
    case 1: return t * kChains * 2.0;
    case 2:
    case 3: return t * kChains;
    case 4: return t * kChains * 2.0;
    case 5:
    case 6: return t * 4.0;
    default: return t * 2.0;
  }
}

cudaError_t launch_probe(int kind, int blocks, int threads, int iters, float* out, int n_out, cudaStream_t st) {
  const size_t smem = (kind == 5 || kind == 6) ? kSharedWords * sizeof(unsigned int) : 0;
  ProbeKernel k = probe_kernel(kind);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<blocks, threads, smem, st>>>(iters, out, n_out);
  return cudaGetLastError();
}

}  // namespace fr
