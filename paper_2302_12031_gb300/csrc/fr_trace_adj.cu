// Adjoint kernel (row a9): reverse mode of the forward trace, recomputing each
// ray's path from its id instead of storing it.
//
// Per ray: the forward code of fr_device.cuh runs again; dL/dE is gathered on
// the nu x nu footprint (kept in registers while the footprint does not move);
// ray_reverse() carries it back through the filter, propagation, Schlick,
// Snell and the normal (and, for point sources, the intersection by the
// implicit function theorem) to the three adjoints (zeta, Zs_bar, Zt_bar); the
// 16 control-point gradients of the ray's knot span are
//   dL/dP_{k+a,l+b} += zeta N_a N_b + Zs_bar N'_a N_b + Zt_bar N_a N'_b
// and are summed in registers while the span does not change, then flushed to a
// CTA-private copy of dL/dP in shared memory, which is added to global memory
// once at the end.
#include "fr_device.cuh"

namespace fr {
namespace {

template <bool DET>
struct GAccT;
template <>
struct GAccT<false> { using type = float; };
template <>
struct GAccT<true> { using type = long long; };

template <bool DET>
struct GradAcc {
  int k, l;
  typename GAccT<DET>::type g[4][4];
};

template <bool DET>
__device__ __forceinline__ void grad_flush(GradAcc<DET>& acc, int ncv, float* sg_f, unsigned long long* sg_q) {
  if (acc.k < 0) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const auto v = acc.g[a][b];
      if (v != 0) {
        const int idx = (acc.k + a) * ncv + acc.l + b;
        if constexpr (DET) atomicAdd(sg_q + idx, (unsigned long long)v);
        else atomicAdd(sg_f + idx, v);
      }
    }
  }
  acc.k = -1;
}

template <int NU, bool DET>
__device__ __forceinline__ void adjoint_ray(const Item& it, const RayFwd& r, const Patch& pc, const float4* sbu,
                                            const float4* sbv, float (&G)[NU][NU], int& gie, int& gje,
                                            GradAcc<DET>& acc, float fixP, float* sg_f, unsigned long long* sg_q,
                                            bool point) {
  Foot<NU> f;
  if (!footprint<NU>(it, r.X, r.Y, f)) return;
  if (f.ie != gie || f.je != gje) {
#pragma unroll
    for (int b = 0; b < NU; ++b)
#pragma unroll
      for (int a = 0; a < NU; ++a) G[b][a] = __ldg(it.dLdE + (size_t)(f.je + b) * it.ncol + f.ie + a);
    gie = f.ie;
    gje = f.je;
  }
  float zeta, Zsb, Ztb;
  ray_reverse<NU>(it, r, f, G, point, pc, &zeta, &Zsb, &Ztb);
  float Nu[4], dNu[4], Nv[4], dNv[4];
  basis_eval(sbu + pc.k * 4, r.s, Nu, dNu);
  basis_eval(sbv + pc.l * 4, r.t, Nv, dNv);
  if (pc.k != acc.k || pc.l != acc.l) {
    grad_flush<DET>(acc, it.ncv, sg_f, sg_q);
    acc.k = pc.k;
    acc.l = pc.l;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc.g[a][b] = 0;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float A = fmaf(zeta, Nu[a], Zsb * dNu[a]);
    const float B = Ztb * Nu[a];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float c = fmaf(A, Nv[b], B * dNv[b]);
      if constexpr (DET) acc.g[a][b] += __float2ll_rn(c * fixP);
      else acc.g[a][b] += c;
    }
  }
}

template <int NU, bool DET>
__device__ void run_adjoint_tiles(const Item& it, const float4* sp, const float4* sbu, const float4* sbv, int t0,
                                  int t1, float zmin, float zmax, float fixP, float* sg_f,
                                  unsigned long long* sg_q, unsigned int* s_cnt) {
  const int R = it.rays_per_lane;
  Patch pc;
  pc.k = -1;
  pc.l = -1;
  GradAcc<DET> acc;
  acc.k = -1;
  float G[NU][NU];
  int gie = -1, gje = -1;
  Counters cnt;
  cnt.clear();
  if (it.kind == FR_SOURCE_COLLIMATED) {
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
    for (int tile = t0; tile < t1; ++tile) {
      const int rg = tile / it.segs, sg = tile - rg * it.segs;
      const int row = it.row_lo + rg * warps + warp;
      if (row >= it.row_hi) continue;
      const int col0 = (sg * 32 + lane) * R;
      for (int j = 0; j < R; ++j) {
        const int col = col0 + j;
        if (col >= it.cols) break;
        const uint64_t id = (uint64_t)row * (uint64_t)it.cols + (uint64_t)col;
        if (id < it.ray_begin || id >= it.ray_end) continue;
        RayFwd r;
        trace_collimated(it, sp, pc, row, col, id, inv_cols, inv_rows, r);
        cnt.add(r.status);
        if (r.status != FR_RAY_ON_SCREEN) continue;
        adjoint_ray<NU, DET>(it, r, pc, sbu, sbv, G, gie, gje, acc, fixP, sg_f, sg_q, false);
      }
    }
  } else {
    const uint64_t per_tile = (uint64_t)blockDim.x * (uint64_t)R;
    for (int tile = t0; tile < t1; ++tile) {
      const uint64_t base = it.ray_begin + (uint64_t)tile * per_tile + threadIdx.x;
      for (int j = 0; j < R; ++j) {
        const uint64_t id = base + (uint64_t)j * blockDim.x;
        if (id >= it.ray_end) break;
        RayFwd r;
        trace_point(it, sp, pc, id, zmin, zmax, r);
        cnt.add(r.status);
        if (r.status != FR_RAY_ON_SCREEN) continue;
        adjoint_ray<NU, DET>(it, r, pc, sbu, sbv, G, gie, gje, acc, fixP, sg_f, sg_q, true);
      }
    }
  }
  grad_flush<DET>(acc, it.ncv, sg_f, sg_q);
  cnt.reduce_into(s_cnt);
}

template <int CAP, bool DET>
__global__ void __launch_bounds__(256) k_adjoint(const __grid_constant__ Launch<CAP> L) {
  int ii = 0;
  while (ii + 1 < L.n_items && (int)blockIdx.x >= L.items[ii].cta_end) ++ii;
  const Item& it = L.items[ii];
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);
  const int np4 = it.nsu * it.nsv * 4;
  float4* sbu = sp + np4;
  float4* sbv = sbu + it.nsu * 4;
  unsigned char* grad_raw = reinterpret_cast<unsigned char*>(sbv + it.nsv * 4);
  float* sg_f = reinterpret_cast<float*>(grad_raw);
  unsigned long long* sg_q = reinterpret_cast<unsigned long long*>(grad_raw);
  for (int q = threadIdx.x; q < np4; q += blockDim.x) sp[q] = it.patch[q];
  for (int q = threadIdx.x; q < it.nsu * 4; q += blockDim.x) sbu[q] = it.basis_u[q];
  for (int q = threadIdx.x; q < it.nsv * 4; q += blockDim.x) sbv[q] = it.basis_v[q];
  const int nctrl = it.ncu * it.ncv;
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) sg_q[q] = 0ull;
    else sg_f[q] = 0.0f;
  }
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  float fixP = 0.0f;
  if constexpr (DET) {
    // Fixed-point scale 2^40 / (max|dL/dE| * flux / pixel area), a power of two.
    const float unit = *it.gmax * it.fixP_unit;
    int e = 0;
    if (unit > 0.0f) frexpf(unit, &e);
    fixP = unit > 0.0f ? ldexpf(1.0f, 40 - e) : 1.0f;
  }
  const float zmin = it.zb[0], zmax = it.zb[1];
  const int ci = (int)blockIdx.x - it.cta_begin, G = it.cta_end - it.cta_begin;
  const int t0 = (int)((long long)it.tiles * ci / G), t1 = (int)((long long)it.tiles * (ci + 1) / G);
  switch (it.nu) {
    case 1: run_adjoint_tiles<1, DET>(it, sp, sbu, sbv, t0, t1, zmin, zmax, fixP, sg_f, sg_q, s_cnt); break;
    case 3: run_adjoint_tiles<3, DET>(it, sp, sbu, sbv, t0, t1, zmin, zmax, fixP, sg_f, sg_q, s_cnt); break;
    default: run_adjoint_tiles<5, DET>(it, sp, sbu, sbv, t0, t1, zmin, zmax, fixP, sg_f, sg_q, s_cnt); break;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) {
      const unsigned long long v = sg_q[q];
      if (v) atomicAdd(it.Pfix + q, v);
    } else {
      const float v = sg_f[q];
      if (v != 0.0f) atomicAdd(it.dLdP + q, v);
    }
  }
  Counters::publish(s_cnt, it.stats);
}

// Deterministic mode: int64 fixed point -> float gradient, with the scale the
// adjoint kernel used (recomputed from the same device value).
__global__ void k_grad_fix_to_float(const __grid_constant__ Item it, int accumulate) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= it.ncu * it.ncv) return;
  const float unit = *it.gmax * it.fixP_unit;
  int e = 0;
  if (unit > 0.0f) frexpf(unit, &e);
  const double inv = unit > 0.0f ? ldexp(1.0, e - 40) : 1.0;
  const float v = (float)((double)(long long)it.Pfix[q] * inv);
  it.dLdP[q] = accumulate ? it.dLdP[q] + v : v;
}

}  // namespace

size_t adj_smem_bytes(const Item& it, bool det) {
  return (size_t)it.nsu * it.nsv * 4 * sizeof(float4) + (size_t)(it.nsu + it.nsv) * 4 * sizeof(float4) +
         (size_t)it.ncu * it.ncv * (det ? 8 : 4);
}

template <int CAP>
cudaError_t launch_adjoint(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st) {
  const int threads = 32 * L.warps;
  if (det) k_adjoint<CAP, true><<<grid, threads, smem, st>>>(L);
  else k_adjoint<CAP, false><<<grid, threads, smem, st>>>(L);
  return cudaGetLastError();
}
template cudaError_t launch_adjoint<1>(const Launch<1>&, int, size_t, bool, cudaStream_t);
template cudaError_t launch_adjoint<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t);

cudaError_t launch_grad_fix_to_float(const Item& it, int accumulate, cudaStream_t st) {
  const int n = it.ncu * it.ncv;
  k_grad_fix_to_float<<<(n + 255) / 256, 256, 0, st>>>(it, accumulate);
  return cudaGetLastError();
}

int adjoint_occupancy(int threads, size_t smem, bool det, bool batch) {
  int n = 0;
  if (batch) {
    if (det) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adjoint<kMaxItems, true>, threads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adjoint<kMaxItems, false>, threads, smem);
  } else {
    if (det) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adjoint<1, true>, threads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adjoint<1, false>, threads, smem);
  }
  return n;
}

// Opt every variant of the kernel in to the largest dynamic shared memory the
// device allows next to the kernel's own static shared memory.
template <class K>
static cudaError_t allow_max_smem(K kernel, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}

cudaError_t configure_adjoint(int optin) {
  cudaError_t e;
  if ((e = allow_max_smem(k_adjoint<1, false>, optin))) return e;
  if ((e = allow_max_smem(k_adjoint<1, true>, optin))) return e;
  if ((e = allow_max_smem(k_adjoint<kMaxItems, false>, optin))) return e;
  return allow_max_smem(k_adjoint<kMaxItems, true>, optin);
}

}  // namespace fr
