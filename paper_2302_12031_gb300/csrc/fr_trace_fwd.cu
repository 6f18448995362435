// Forward trace kernel (rows a1-a7) and the per-ray debug kernel.
//
// Schedule: each CTA works on one lens (item) and on a contiguous range of that
// item's tiles, so its rays come from one compact part of the aperture.
//  - collimated: a tile is `warps` consecutive grid rows x (32 * R) columns;
//    lane l of warp w traces the R consecutive rays (row w, columns l*R ...);
//  - point: a tile is blockDim * R consecutive ray ids.
// Each lane keeps the nu x nu footprint of its last ray in registers and adds
// the next ray there while the footprint does not move; it flushes the
// registers (with atomics) when it does. Consecutive collimated rays usually
// share a pixel, so most rays cost no atomic at all. The flush goes to a
// privatised histogram in shared memory when the extended grid fits, else
// straight to global memory.
#include "fr_device.cuh"

namespace fr {
namespace {

template <bool DET>
struct AccT;
template <>
struct AccT<false> { using type = float; };
template <>
struct AccT<true> { using type = long long; };

struct Bbox {
  int imin, imax, jmin, jmax;
};

struct Target {
  bool smem;
  int ncol;
  float* sh_f;
  unsigned long long* sh_q;
  float* gl_f;
  unsigned long long* gl_q;
};

template <int NU, bool DET>
struct FootAcc {
  int ie, je;
  typename AccT<DET>::type v[NU][NU];
};

template <int NU, bool DET>
__device__ __forceinline__ void acc_flush(FootAcc<NU, DET>& acc, const Target& tg, Bbox& bb) {
  if (acc.ie < 0) return;
  bb.imin = min(bb.imin, acc.ie);
  bb.imax = max(bb.imax, acc.ie);
  bb.jmin = min(bb.jmin, acc.je);
  bb.jmax = max(bb.jmax, acc.je);
#pragma unroll
  for (int b = 0; b < NU; ++b) {
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      const auto val = acc.v[b][a];
      if (val != 0) {
        const int idx = (acc.je + b) * tg.ncol + acc.ie + a;
        if constexpr (DET) {
          if (tg.smem) atomicAdd(tg.sh_q + idx, (unsigned long long)val);
          else atomicAdd(tg.gl_q + idx, (unsigned long long)val);
        } else {
          if (tg.smem) atomicAdd(tg.sh_f + idx, val);
          else atomicAdd(tg.gl_f + idx, val);
        }
      }
    }
  }
  acc.ie = -1;
}

template <int NU, bool DET>
__device__ __forceinline__ void deposit(const Item& it, const RayFwd& r, const Target& tg, FootAcc<NU, DET>& acc,
                                        Bbox& bb) {
  Foot<NU> f;
  if (!footprint<NU>(it, r.X, r.Y, f)) return;
  if (f.ie != acc.ie || f.je != acc.je) {
    acc_flush<NU, DET>(acc, tg, bb);
    acc.ie = f.ie;
    acc.je = f.je;
#pragma unroll
    for (int b = 0; b < NU; ++b)
#pragma unroll
      for (int a = 0; a < NU; ++a) acc.v[b][a] = 0;
  }
  // E_ij += w F_ij / (w_x w_y), F_ij = (f_i / S_x) (f_j / S_y).
  const float K = r.w * it.inv_area;
  float kx[NU], ky[NU];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    kx[a] = f.fx[a] * f.rsx * K;
    ky[a] = f.fy[a] * f.rsy;
  }
#pragma unroll
  for (int b = 0; b < NU; ++b) {
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      const float c = kx[a] * ky[b];
      if constexpr (DET) acc.v[b][a] += __float2ll_rn(c * it.fixE);
      else acc.v[b][a] += c;
    }
  }
}

template <int NU, bool DET>
__device__ void run_tiles(const Item& it, const float4* sp, const Target& tg, int t0, int t1, float zmin, float zmax,
                          Counters& cnt, Bbox& bb) {
  const int R = it.rays_per_lane;
  Patch pc;
  pc.k = -1;
  pc.l = -1;
  FootAcc<NU, DET> acc;
  acc.ie = -1;
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
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET>(it, r, tg, acc, bb);
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
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET>(it, r, tg, acc, bb);
      }
    }
  }
  acc_flush<NU, DET>(acc, tg, bb);
}

template <int CAP, bool DET>
__global__ void __launch_bounds__(256) k_forward(const __grid_constant__ Launch<CAP> L) {
  int ii = 0;
  while (ii + 1 < L.n_items && (int)blockIdx.x >= L.items[ii].cta_end) ++ii;
  const Item& it = L.items[ii];
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);
  const int np4 = it.nsu * it.nsv * 4;
  for (int q = threadIdx.x; q < np4; q += blockDim.x) sp[q] = it.patch[q];
  unsigned char* hist_raw = smem + (size_t)np4 * sizeof(float4);
  const int ncell = it.ncol * it.nrow;
  Target tg;
  tg.smem = it.smem_hist != 0;
  tg.ncol = it.ncol;
  tg.sh_f = reinterpret_cast<float*>(hist_raw);
  tg.sh_q = reinterpret_cast<unsigned long long*>(hist_raw);
  tg.gl_f = it.E;
  tg.gl_q = it.Efix;
  if (tg.smem) {
    if constexpr (DET) {
      for (int q = threadIdx.x; q < ncell; q += blockDim.x) tg.sh_q[q] = 0ull;
    } else {
      for (int q = threadIdx.x; q < ncell; q += blockDim.x) tg.sh_f[q] = 0.0f;
    }
  }
  __shared__ int s_bb[4];
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  if (threadIdx.x < 4) s_bb[threadIdx.x] = (threadIdx.x & 1) ? -1 : 0x7fffffff;
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const float zmin = it.zb[0], zmax = it.zb[1];
  const int ci = (int)blockIdx.x - it.cta_begin, G = it.cta_end - it.cta_begin;
  const int t0 = (int)((long long)it.tiles * ci / G), t1 = (int)((long long)it.tiles * (ci + 1) / G);
  Counters cnt;
#pragma unroll
  for (int s = 0; s < FR_RAY_NCAUSES; ++s) cnt.n[s] = 0u;
  Bbox bb{0x7fffffff, -1, 0x7fffffff, -1};
  switch (it.nu) {
    case 1: run_tiles<1, DET>(it, sp, tg, t0, t1, zmin, zmax, cnt, bb); break;
    case 3: run_tiles<3, DET>(it, sp, tg, t0, t1, zmin, zmax, cnt, bb); break;
    default: run_tiles<5, DET>(it, sp, tg, t0, t1, zmin, zmax, cnt, bb); break;
  }
  cnt.reduce_into(s_cnt);
  if (tg.smem && bb.imax >= 0) {
    atomicMin(&s_bb[0], bb.imin);
    atomicMax(&s_bb[1], bb.imax);
    atomicMin(&s_bb[2], bb.jmin);
    atomicMax(&s_bb[3], bb.jmax);
  }
  __syncthreads();
  if (tg.smem && s_bb[1] >= 0) {
    // Flush the touched window of the privatised histogram.
    const int nu = it.nu;
    const int c0 = s_bb[0], c1 = s_bb[1] + nu - 1, r0 = s_bb[2], r1 = s_bb[3] + nu - 1;
    const int wcols = c1 - c0 + 1, n = wcols * (r1 - r0 + 1);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int rr = r0 + q / wcols, cc = c0 + q % wcols;
      const int idx = rr * it.ncol + cc;
      if constexpr (DET) {
        const unsigned long long v = tg.sh_q[idx];
        if (v) atomicAdd(tg.gl_q + idx, v);
      } else {
        const float v = tg.sh_f[idx];
        if (v != 0.0f) atomicAdd(tg.gl_f + idx, v);
      }
    }
  }
  Counters::publish(s_cnt, it.stats);
}

// One thread per ray: the full record of rays [ray_begin, ray_end).
__global__ void k_debug(const __grid_constant__ Item it, fr_ray_record* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t id = it.ray_begin + i;
  if (id >= it.ray_end) return;
  Patch pc;
  pc.k = -1;
  pc.l = -1;
  RayFwd r;
  r.status = FR_RAY_ON_SCREEN;
  r.u = r.v = r.s = r.t = r.x = r.y = r.z = r.dx = r.dy = r.dz = 0.0f;
  r.tx = r.ty = r.tz = r.w = r.X = r.Y = r.tstar = 0.0f;
  r.iters = 0;
  if (it.kind == FR_SOURCE_COLLIMATED) {
    const int row = (int)(id / (uint64_t)it.cols), col = (int)(id % (uint64_t)it.cols);
    trace_collimated(it, it.patch, pc, row, col, id, 1.0f / (float)it.cols, 1.0f / (float)it.rows, r);
  } else {
    trace_point(it, it.patch, pc, id, it.zb[0], it.zb[1], r);
  }
  fr_ray_record rec;
  rec.status = r.status;
  rec.span_i = pc.k >= 0 ? pc.k + 3 : -1;
  rec.span_j = pc.l >= 0 ? pc.l + 3 : -1;
  rec.newton_iters = r.iters;
  rec.u = r.u;
  rec.v = r.v;
  rec.x = r.x;
  rec.y = r.y;
  rec.z = r.z;
  rec.dx = r.dx;
  rec.dy = r.dy;
  rec.dz = r.dz;
  rec.tx = r.tx;
  rec.ty = r.ty;
  rec.tz = r.tz;
  rec.X = r.X;
  rec.Y = r.Y;
  rec.w = r.w;
  rec.t = r.tstar;
  out[i] = rec;
}

}  // namespace

size_t fwd_smem_bytes(const Item& it, bool det) {
  size_t b = (size_t)it.nsu * it.nsv * 4 * sizeof(float4);
  if (it.smem_hist) b += (size_t)it.ncol * it.nrow * (det ? 8 : 4);
  return b;
}

template <int CAP>
cudaError_t launch_forward(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st) {
  const int threads = 32 * L.warps;
  if (det) k_forward<CAP, true><<<grid, threads, smem, st>>>(L);
  else k_forward<CAP, false><<<grid, threads, smem, st>>>(L);
  return cudaGetLastError();
}
template cudaError_t launch_forward<1>(const Launch<1>&, int, size_t, bool, cudaStream_t);
template cudaError_t launch_forward<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t);

cudaError_t launch_debug(const Item& it, fr_ray_record* out, cudaStream_t st) {
  const uint64_t n = it.ray_end - it.ray_begin;
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  const unsigned int blocks = (unsigned int)((n + threads - 1) / threads);
  k_debug<<<blocks, threads, 0, st>>>(it, out);
  return cudaGetLastError();
}

int forward_occupancy(int threads, size_t smem, bool det, bool batch) {
  int n = 0;
  if (batch) {
    if (det) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward<kMaxItems, true>, threads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward<kMaxItems, false>, threads, smem);
  } else {
    if (det) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward<1, true>, threads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward<1, false>, threads, smem);
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

cudaError_t configure_forward(int optin) {
  cudaError_t e;
  if ((e = allow_max_smem(k_forward<1, false>, optin))) return e;
  if ((e = allow_max_smem(k_forward<1, true>, optin))) return e;
  if ((e = allow_max_smem(k_forward<kMaxItems, false>, optin))) return e;
  return allow_max_smem(k_forward<kMaxItems, true>, optin);
}

}  // namespace fr
