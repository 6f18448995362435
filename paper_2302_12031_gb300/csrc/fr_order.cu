// Coherent order of point-source rays (fr_ray_order).
//
// Point-source directions are drawn per ray id (Sec. 2.2.1), so consecutive ids
// meet the lens at unrelated places: a lane's consecutive rays rarely share a
// knot span or a pixel, and the warps' Newton iterations diverge. A counting
// sort of the ids by (source, cell of the entry plane where the ray meets it)
// gives the traces an order in which neighbouring positions are neighbouring
// rays, with the rays that miss the aperture (most of a wide cone) last: the
// traces split only the others over their lanes, so no warp idles on misses.
// The key is not the entry point itself but its image on the plane of the
// mean control height, reached along the refracted direction: the hit of a
// ray on the exit face lies close to that image, the entry point up to the
// glass's thickness times the slope of the ray away. The cells subdivide the
// knot spans there (m x m cells per span, spans in row order, cells in Z order
// within a span), so a run of positions stays in one span: the adjoint sums a
// lane's gradient terms per span in registers and writes them out when the
// span changes. The key depends on the control heights through their mean
// only, and only for coherence: any permutation is a correct order.
#include "fr_device.cuh"

namespace fr {
namespace {

// Bits 0..7 of x spread to the even bits 0..14.
__device__ __forceinline__ uint32_t spread_bits(uint32_t x) {
  x &= 0xffu;
  x = (x | (x << 4)) & 0x0f0fu;
  x = (x | (x << 2)) & 0x3333u;
  x = (x | (x << 1)) & 0x5555u;
  return x;
}

// Source index x (nsu nsv m^2 + 1) + the index of the cell of ray `id`: (knot
// span row x nsu + span column) m^2 + the Z-order index of the m x m cell
// within the span, at the point where the refracted ray meets the plane
// z_in + h (h the mean glass thickness), or nsu nsv m^2 where that point lies
// outside the aperture (rays that mostly leave the glass through its side);
// n_src (nsu nsv m^2 + 1) (the last key) for a ray that misses the aperture.
// The miss test is the trace's with a margin of 1e-5 relative, so a ray put
// with the misses misses in the trace too.
__device__ __forceinline__ uint32_t ray_key(const Item& it, uint64_t id, int m, float h) {
  float sx, sy, d0x, d0y, d0z, omc, sphi;
  source_ray(it, id, &sx, &sy, &d0x, &d0y, &d0z, &omc, &sphi);
  const float tau = __fdiv_rn(it.z_in - it.pz, d0z);
  const float ox = fmaf(tau, d0x, sx), oy = fmaf(tau, d0y, sy);
  const uint32_t nsrc = (uint32_t)(it.gnx * it.gny);
  const uint32_t cells = (uint32_t)(it.nsu * it.nsv) * (uint32_t)(m * m), per_src = cells + 1u;
  if (!(tau > 0.0f) || fabsf(ox) > __fmul_rn(it.rx, 1.00001f) || fabsf(oy) > __fmul_rn(it.ry, 1.00001f))
    return nsrc * per_src;
  // the in-glass direction is (d0x, d0y, .) / n_glass with z part
  // sqrt(1 - sin^2 / n_glass^2): h / dz times its lateral part
  const float eta = __fdiv_rn(1.0f, it.n_glass);
  const float dz = __fsqrt_rn(__fadd_rn(1.0f, -__fmul_rn(__fmul_rn(eta, eta), __fmul_rn(sphi, sphi))));
  const float g = __fdiv_rn(__fmul_rn(h, eta), dz);
  const float px = fmaf(g, d0x, ox), py = fmaf(g, d0y, oy);
  uint32_t src = 0;
  if (nsrc > 1) src = min((uint32_t)(id / it.per_src), nsrc - 1);
  if (!(fabsf(px) <= it.rx && fabsf(py) <= it.ry)) return src * per_src + cells;
  // position in knot-span units, u nsu with u = x / (2 rx) + 1/2
  const float us = __fmul_rn(__fdiv_rn(px, it.rx) + 1.0f, 0.5f * (float)it.nsu);
  const float vs = __fmul_rn(__fdiv_rn(py, it.ry) + 1.0f, 0.5f * (float)it.nsv);
  const int k = min(max((int)us, 0), it.nsu - 1), l = min(max((int)vs, 0), it.nsv - 1);
  const int cx = min(max((int)__fmul_rn(us - (float)k, (float)m), 0), m - 1);
  const int cy = min(max((int)__fmul_rn(vs - (float)l, (float)m), 0), m - 1);
  const uint32_t cell = (uint32_t)(l * it.nsu + k) * (uint32_t)(m * m) +
                        (spread_bits((uint32_t)cx) | (spread_bits((uint32_t)cy) << 1));
  return src * per_src + cell;
}

// Mean control height of the exit net minus z_in (0 if not positive), the
// same in every CTA of both passes: warp 0 sums in a fixed order.
__device__ float nominal_thickness(const Item& it) {
  __shared__ float s_h;
  if (threadIdx.x < 32) {
    const int n = it.ncu * it.ncv;
    float sum = 0.0f;
    for (int q = (int)threadIdx.x; q < n; q += 32) sum = __fadd_rn(sum, __ldg(it.ctrl + q));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
    if (threadIdx.x == 0) s_h = fmaxf(__fadd_rn(__fdiv_rn(sum, (float)n), -it.z_in), 0.0f);
  }
  __syncthreads();
  return s_h;
}

// Counts the rays per key and keeps each ray's key for the scatter pass.
__global__ void __launch_bounds__(256) k_order_count(const __grid_constant__ Item it, int m, uint32_t* counts,
                                                     uint32_t* keys) {
  const float h = nominal_thickness(it);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < it.n_rays; id += stride) {
    const uint32_t k = ray_key(it, id, m, h);
    keys[id] = k;
    atomicAdd(counts + k, 1u);
  }
}

// Exclusive prefix sum of counts[0..n) in place, one CTA of 1024 threads: each
// thread sums a contiguous chunk, the CTA scans the chunk sums, each thread
// writes its chunk's prefixes. The prefix of the last key (the misses) is the
// number of rays that meet the aperture: it goes to *hits (when given).
__global__ void __launch_bounds__(1024) k_order_scan(uint32_t* counts, uint64_t n, uint32_t* hits, uint32_t all) {
  __shared__ uint32_t s_warp[32];
  const uint64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = min(n, chunk * threadIdx.x), hi = min(n, lo + chunk);
  uint32_t sum = 0;
  for (uint64_t i = lo; i < hi; ++i) sum += counts[i];
  // inclusive scan of the thread sums: within warps, then across warp totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;   // inclusive over warps 0..lane
  }
  __syncthreads();
  uint32_t run = incl - sum + (warp > 0 ? s_warp[warp - 1] : 0u);   // exclusive prefix of this chunk
  for (uint64_t i = lo; i < hi; ++i) {
    const uint32_t c = counts[i];
    counts[i] = run;
    if (i == n - 1 && hits) *hits = all ? all : run;
    run += c;
  }
}

// The same scan for many keys, in three launches: the sum of every tile of
// kScanTile counts (k_scan_partial), the scan of those sums (k_order_scan on
// one CTA), then each tile's own scan from its offset (k_scan_apply).
constexpr uint64_t kScanTile = 8192;   // 1024 threads x 8 counts

__device__ __forceinline__ uint32_t block_sum_1024(uint32_t v, uint32_t* s_warp) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? s_warp[threadIdx.x] : 0u;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // in thread 0
}

__global__ void __launch_bounds__(1024) k_scan_partial(const uint32_t* counts, uint64_t n, uint32_t* partial) {
  __shared__ uint32_t s_warp[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t i = base + threadIdx.x + 1024u * j;
    if (i < n) v += counts[i];
  }
  const uint32_t t = block_sum_1024(v, s_warp);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_scan_apply(uint32_t* counts, uint64_t n, const uint32_t* partial,
                                                     uint32_t* hits, uint32_t all) {
  __shared__ uint32_t s_warp[32];
  const uint64_t lo = min(n, (uint64_t)blockIdx.x * kScanTile + 8u * threadIdx.x), hi = min(n, lo + 8);
  uint32_t c[8], sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j] = lo + j < hi ? counts[lo + j] : 0u;
    sum += c[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;   // inclusive over warps 0..lane
  }
  __syncthreads();
  uint32_t run = partial[blockIdx.x] + incl - sum + (warp > 0 ? s_warp[warp - 1] : 0u);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t i = lo + j;
    if (i < hi) {
      counts[i] = run;
      if (i == n - 1) *hits = all ? all : run;
      run += c[j];
    }
  }
}

__global__ void __launch_bounds__(256) k_order_scatter(const __grid_constant__ Item it, const uint32_t* keys,
                                                       uint32_t* cursor, uint32_t* order) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < it.n_rays; id += stride) {
    // the counting pass's key; the bound only guards memory
    const uint32_t pos = atomicAdd(cursor + keys[id], 1u);
    if (pos < it.n_rays) order[pos] = (uint32_t)id;
  }
}

}  // namespace

// Cells per knot span side m: a power of two in 1..128 with 16 or more of one
// source's rays per cell (finer cells keep the rays whose hit lies across a
// knot line from the projected point together in the order: on the 16M-ray
// point source the adjoint took 667 us with 16 rays per cell, 695 with 128).
int ray_order_grid(const Item& it) {
  const uint64_t per_span = it.n_rays / (uint64_t)(it.gnx * it.gny) / (uint64_t)(it.nsu * it.nsv);
  int m = 1;
  while (m < 128 && (uint64_t)(2 * m) * (uint64_t)(2 * m) * 16u <= per_span) m *= 2;
  return m;
}

uint64_t ray_order_keys(const Item& it, int m) {
  return (uint64_t)(it.gnx * it.gny) * ((uint64_t)(it.nsu * it.nsv) * (uint64_t)(m * m) + 1) + 1;
}

uint64_t ray_order_scratch_words(const Item& it, int m) {
  return (ray_order_keys(it, m) + kScanTile - 1) / kScanTile;
}

cudaError_t launch_ray_order(const Item& it, int m, uint32_t* counts, uint32_t* keys, uint32_t* partial,
                             uint32_t* order, cudaStream_t st) {
  const uint64_t nk = ray_order_keys(it, m);
  cudaError_t e = cudaMemsetAsync(counts, 0, nk * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const uint64_t want = (it.n_rays + 255) / 256;
  const unsigned int blocks = (unsigned int)(want < 4096 ? want : 4096);
  k_order_count<<<blocks, 256, 0, st>>>(it, m, counts, keys);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // a freeform entry face decides the aperture in the trace: every position is traced
  const uint32_t all = it.two_face ? (uint32_t)it.n_rays : 0u;
  const uint64_t tiles = (nk + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_order_scan<<<1, 1024, 0, st>>>(counts, nk, order + it.n_rays, all);
  } else {
    k_scan_partial<<<(unsigned int)tiles, 1024, 0, st>>>(counts, nk, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_order_scan<<<1, 1024, 0, st>>>(partial, tiles, nullptr, 0u);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan_apply<<<(unsigned int)tiles, 1024, 0, st>>>(counts, nk, partial, order + it.n_rays, all);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scatter<<<blocks, 256, 0, st>>>(it, keys, counts, order);
  return cudaGetLastError();
}

}  // namespace fr
