// Coherent order of point-source rays (fr_ray_order).
//
// Point-source directions are drawn per ray id (Sec. 2.2.1), so consecutive ids
// meet the lens at unrelated places: a lane's consecutive rays rarely share a
// knot span or a pixel, and the warps' Newton iterations diverge. A counting
// sort of the ids by (source, cell of the entry plane where the ray meets it)
// gives the traces an order in which neighbouring positions are neighbouring
// rays, with the rays that miss the aperture (most of a wide cone) last: the
// traces split only the others over their lanes, so no warp idles on misses.
// The key is computed from the source sampling and the flat entry plane alone,
// so it does not depend on the control heights.
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

// Source index x G^2 + the Z-order index of the G x G aperture cell where ray
// `id` meets the entry plane; n_src G^2 (the last key) for a ray that misses the
// aperture. The miss test is the trace's with a margin of 1e-5 relative, so a
// ray put with the misses misses in the trace too.
__device__ __forceinline__ uint32_t ray_key(const Item& it, uint64_t id, int G) {
  float sx, sy, d0x, d0y, d0z, omc, sphi;
  source_ray(it, id, &sx, &sy, &d0x, &d0y, &d0z, &omc, &sphi);
  const float tau = __fdiv_rn(it.z_in - it.pz, d0z);
  const float ox = fmaf(tau, d0x, sx), oy = fmaf(tau, d0y, sy);
  const uint32_t nsrc = (uint32_t)(it.gnx * it.gny);
  if (!(tau > 0.0f) || fabsf(ox) > __fmul_rn(it.rx, 1.00001f) || fabsf(oy) > __fmul_rn(it.ry, 1.00001f))
    return nsrc * (uint32_t)(G * G);
  const float g = 0.5f * (float)G;
  const int cx = min(max((int)__fmul_rn(__fdiv_rn(ox, it.rx) + 1.0f, g), 0), G - 1);
  const int cy = min(max((int)__fmul_rn(__fdiv_rn(oy, it.ry) + 1.0f, g), 0), G - 1);
  const uint32_t cell = spread_bits((uint32_t)cx) | (spread_bits((uint32_t)cy) << 1);
  uint32_t src = 0;
  if (nsrc > 1) src = min((uint32_t)(id / it.per_src), nsrc - 1);
  return src * (uint32_t)(G * G) + cell;
}

__global__ void __launch_bounds__(256) k_order_count(const __grid_constant__ Item it, int G, uint32_t* counts) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < it.n_rays; id += stride)
    atomicAdd(counts + ray_key(it, id, G), 1u);
}

// Exclusive prefix sum of counts[0..n) in place, one CTA of 1024 threads: each
// thread sums a contiguous chunk, the CTA scans the chunk sums, each thread
// writes its chunk's prefixes. The prefix of the last key (the misses) is the
// number of rays that meet the aperture: it goes to *hits.
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
    if (i == n - 1) *hits = all ? all : run;
    run += c;
  }
}

__global__ void __launch_bounds__(256) k_order_scatter(const __grid_constant__ Item it, int G, uint32_t* cursor,
                                                       uint32_t* order) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < it.n_rays; id += stride) {
    // The key is the counting pass's to the bit (the same code, with no
    // contractible a*b+c left in it); the bound only guards memory.
    const uint32_t pos = atomicAdd(cursor + ray_key(it, id, G), 1u);
    if (pos < it.n_rays) order[pos] = (uint32_t)id;
  }
}

}  // namespace

// About 128 rays per cell of one source's grid, G a power of two in 1..128.
int ray_order_grid(const Item& it) {
  const uint64_t per_src = it.n_rays / (uint64_t)(it.gnx * it.gny);
  int G = 1;
  while (G < 128 && (uint64_t)(2 * G) * (uint64_t)(2 * G) * 128u <= per_src) G *= 2;
  return G;
}

uint64_t ray_order_keys(const Item& it, int G) { return (uint64_t)(it.gnx * it.gny) * (uint64_t)(G * G) + 1; }

cudaError_t launch_ray_order(const Item& it, int G, uint32_t* counts, uint32_t* order, cudaStream_t st) {
  const uint64_t nk = ray_order_keys(it, G);
  cudaError_t e = cudaMemsetAsync(counts, 0, nk * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const uint64_t want = (it.n_rays + 255) / 256;
  const unsigned int blocks = (unsigned int)(want < 4096 ? want : 4096);
  k_order_count<<<blocks, 256, 0, st>>>(it, G, counts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // a freeform entry face decides the aperture in the trace: every position is traced
  k_order_scan<<<1, 1024, 0, st>>>(counts, nk, order + it.n_rays, it.two_face ? (uint32_t)it.n_rays : 0u);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scatter<<<blocks, 256, 0, st>>>(it, G, counts, order);
  return cudaGetLastError();
}

}  // namespace fr
