// Forward-mode trace kernel: directional derivatives (dE/dP^z) dP_k of the
// irradiance for a few directions dP_k at once — for one control point, the
// derivative maps of Sec. 3.1.
//
// Each CTA builds the lens tables (as the forward kernel) and a bit mask per
// knot-span patch of the directions that move one of its 16 control points.
// Every lane takes an equal run of consecutive ray ids; a ray whose patch no
// direction moves stops before the trace (collimated: the patch follows from
// the ray's grid cell) or right after it (point source). For the others, the tangents of the
// hit height and slopes, sum_ab N_a N_b dP, sum_ab N'_a N_b dP and
// sum_ab N_a N'_b dP (for a point source also the hit's shift along the ray by
// the implicit function theorem), go through ray_tangent, and
//   dE_ij += (dw F_ij + w (dF_ij/dX dX + dF_ij/dY dY)) / (w_x w_y)
// is added to the nu x nu footprint of direction k with global atomics (for a
// single direction summed first in registers while a lane's footprint stays).
#include "fr_device.cuh"

namespace fr {
namespace {

// Adds a lane's register footprint to the map (one direction) and clears it.
template <int NU>
__device__ __forceinline__ void flush_acc(float (&acc)[NU][NU], int ie, int je, float* dE, int ncol) {
  if (ie < 0) return;
#pragma unroll
  for (int b = 0; b < NU; ++b)
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      if (acc[b][a] != 0.0f) atomicAdd(dE + (size_t)(je + b) * ncol + ie + a, acc[b][a]);
      acc[b][a] = 0.0f;
    }
}

template <int NU>
__global__ void __launch_bounds__(256, 2) k_tangent(const __grid_constant__ Item it, int warps,
                                                    const float* __restrict__ dP, int n_dirs,
                                                    float* __restrict__ dE) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = carve_exit(smem, it);
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem + ((lens_smem_bytes(it.nsu, it.nsv, needs_hull(it)) + 15) & ~(size_t)15));
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  const int nctrl = it.ncu * it.ncv;
  for (int p = threadIdx.x; p < it.nsu * it.nsv; p += blockDim.x) {
    const int k = p / it.nsv, l = p - k * it.nsv;
    uint32_t m = 0u;
    for (int q = 0; q < n_dirs; ++q) {
      const float* P = dP + (size_t)q * nctrl + k * it.ncv + l;
      bool any = false;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) any |= __ldg(P + a * it.ncv + b) != 0.0f;
      if (any) m |= 1u << q;
    }
    s_mask[p] = m;
  }
  // Collimated rays without per-cause counts: only the grid cells over the
  // bounding box of the patches that some direction moves are traced, split
  // evenly over all lanes (so a direction local to a few patches costs only
  // their rays). The box is the same in every CTA.
  __shared__ int s_box[4];
  const bool coll = it.kind == FR_SOURCE_COLLIMATED;
  const bool boxed = coll && !it.stats;
  if (boxed) {
    if (threadIdx.x == 0) {
      s_box[0] = s_box[2] = 1 << 30;
      s_box[1] = s_box[3] = -1;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < it.nsu * it.nsv; p += blockDim.x) {
      if (s_mask[p]) {
        const int k = p / it.nsv, l = p - k * it.nsv;
        atomicMin(&s_box[0], k);
        atomicMax(&s_box[1], k);
        atomicMin(&s_box[2], l);
        atomicMax(&s_box[3], l);
      }
    }
  }
  build_lens_tables(it, ls);   // ends with __syncthreads

  const size_t cells = (size_t)it.ncol * it.nrow;
  const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
  RayCount cnt{0u};
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  uint64_t a0, a1;
  uint32_t c0 = 0, bw = 1, r0 = 0;
  if (boxed) {
    if (s_box[1] < 0) return;   // no direction moves any patch: dE = 0
    // grid cells [c0, c1) x [r0, r1) whose u (v) interval meets the box's patches
    c0 = (uint32_t)(((uint64_t)s_box[0] * it.cols) / it.nsu);
    const uint64_t c1w = ((uint64_t)(s_box[1] + 1) * it.cols + it.nsu - 1) / it.nsu;
    const uint32_t c1 = (uint32_t)(c1w < (uint64_t)it.cols ? c1w : (uint64_t)it.cols);
    r0 = (uint32_t)(((uint64_t)s_box[2] * it.rows) / it.nsv);
    const uint64_t r1w = ((uint64_t)(s_box[3] + 1) * it.rows + it.nsv - 1) / it.nsv;
    const uint32_t r1 = (uint32_t)(r1w < (uint64_t)it.rows ? r1w : (uint64_t)it.rows);
    bw = c1 - c0;
    const uint64_t V = (uint64_t)bw * (r1 - r0);
    const uint64_t W = (uint64_t)(it.cta_end - it.cta_begin) * (uint64_t)warps;
    const uint64_t gw = (uint64_t)((int)blockIdx.x - it.cta_begin) * (uint64_t)warps + (threadIdx.x >> 5);
    const uint64_t w0 = V * gw / W, w1 = V * (gw + 1) / W;
    const uint64_t lane = threadIdx.x & 31;
    a0 = w0 + (w1 - w0) * lane / 32;
    a1 = w0 + (w1 - w0) * (lane + 1) / 32;
  } else {
    lane_range(it, warps, &a0, &a1);
  }
  constexpr int NA = NU <= 5 ? NU : 1;   // register footprint (unused for larger filters)
  float acc[NA][NA];
#pragma unroll
  for (int b = 0; b < NA; ++b)
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[b][a] = 0.0f;
  int acc_ie = -1, acc_je = -1;
  for (uint64_t j = a0; j < a1; ++j) {
    RayFwd r;
    uint32_t m;
    uint64_t id = j;
    if (boxed) {
      const uint64_t rr = j / bw;
      id = (uint64_t)(r0 + rr) * it.cols + (c0 + (j - rr * bw));
      if (id < it.ray_begin || id >= it.ray_end) continue;
    }
    if (coll) {
      // A collimated ray's patch is known before the trace: rays on patches no
      // direction moves contribute nothing and are only counted.
      const uint32_t row = (uint32_t)(id / (uint64_t)it.cols), col = (uint32_t)(id % (uint64_t)it.cols);
      float ja = 0.5f, jb = 0.5f;
      if (it.jitter) {
        const uint2 w = philox_ray_words(it.seed, id);
        ja = unit23(w.x);
        jb = unit23(w.y);
      }
      const float u = ((float)col + ja) * inv_cols, v = ((float)row + jb) * inv_rows;
      locate(u, it.nsu, &r.k, &r.s);
      locate(v, it.nsv, &r.l, &r.t);
      m = s_mask[r.k * it.nsv + r.l];
      if (m == 0u && !cnt_dst) continue;
      float Z, Zs, Zt;
      patch_eval(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Z, &Zs, &Zt);
      collimated_at(it, u, v, fmaf(2.0f, v, -1.0f) * it.ry, Z, Zs, Zt, r);
    } else {
      float zmin, zmax;
      zbounds(ls, &zmin, &zmax);
      if (it.order) id = __ldg(it.order + j);
      trace_point<true>(it, ls, id, zmin, zmax, r);
      m = 0u;
      if (r.status == FR_RAY_ON_SCREEN) {
        m = s_mask[r.k * it.nsv + r.l];
        if (it.mesh_nu > 0) m |= s_mask[(r.mK / it.mesh_nu) * it.nsv + r.mL / it.mesh_nv];
      }
    }
    cnt.add(r.status, cnt_dst);
    if (r.status != FR_RAY_ON_SCREEN || m == 0u) continue;
    Foot<NU> f;
    if (!footprint_scalar<NU>(it, r.X, r.Y, f)) continue;
    float Nu[4], dNu[4], Nv[4], dNv[4];
    basis_eval(ls.bu + r.k * 4, r.s, Nu, dNu);
    basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
    float Fx[NU], Fy[NU], gx[NU], gy[NU];
    filter_grad<NU>(it, f, Fx, Fy, gx, gy);
    // Point source: the slopes' change along the ray (second derivatives).
    float slope_s = 0.0f, slope_t = 0.0f, inv_gp = 0.0f;
    if (!coll) {
      float Zss, Zst, Ztt;
      patch_eval2(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Zss, &Zst, &Ztt);
      const float dsdt = r.dx * (0.5f / it.rx) * (float)it.nsu;
      const float dtdt = r.dy * (0.5f / it.ry) * (float)it.nsv;
      slope_s = fmaf(Zss, dsdt, Zst * dtdt);
      slope_t = fmaf(Zst, dsdt, Ztt * dtdt);
      inv_gp = 1.0f / r.gp;
    }
    float W[4][4];
    int kt = 0, lt = 0;
    if (!coll && it.mesh_nu > 0) mesh_vertex_weights(it, ls, r, W, &kt, &lt);
    const float K = r.w * it.inv_area;
    while (m) {
      const int q = __ffs(m) - 1;
      m &= m - 1u;
      const float* P = dP + (size_t)q * nctrl + r.k * it.ncv + r.l;
      float dZ = 0.0f, dZs = 0.0f, dZt = 0.0f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        float c = 0.0f, ct = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float v = __ldg(P + a * it.ncv + b);
          c = fmaf(Nv[b], v, c);
          ct = fmaf(dNv[b], v, ct);
        }
        dZ = fmaf(Nu[a], c, dZ);
        dZs = fmaf(dNu[a], c, dZs);
        dZt = fmaf(Nu[a], ct, dZt);
      }
      RayTan tg;
      if (coll) {
        tg = ray_tangent<true>(it, r, 0.0f, 0.0f, dZ, dZs, dZt);
      } else {
        // f(t*, P) = 0: dt* = -dZ / f'(t*); the hit moves along the ray. On the
        // triangle mesh the hit height moves with the triangle's vertices.
        if (it.mesh_nu > 0) {
          const float* Pt = dP + (size_t)q * nctrl + kt * it.ncv + lt;
          dZ = 0.0f;
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) dZ = fmaf(W[a][b], __ldg(Pt + a * it.ncv + b), dZ);
        }
        const float dt = -dZ * inv_gp;
        tg = ray_tangent<false>(it, r, r.dx * dt, r.dy * dt, r.dz * dt, fmaf(slope_s, dt, dZs),
                                fmaf(slope_t, dt, dZt));
      }
      const float cw = tg.dw * it.inv_area, cx = K * tg.dX, cy = K * tg.dY;
      if (NU <= 5 && n_dirs == 1) {
        // One direction: consecutive rays of a lane mostly share a footprint;
        // sum them in registers and flush when the footprint moves (small
        // footprints only: nu^2 registers).
        if (f.ie != acc_ie || f.je != acc_je) {
          flush_acc<NA>(acc, acc_ie, acc_je, dE, it.ncol);
          acc_ie = f.ie;
          acc_je = f.je;
        }
#pragma unroll
        for (int b = 0; b < NA; ++b) {
          const float rb = cw * Fy[b], sb = cx * Fy[b], tb = cy * gy[b];
#pragma unroll
          for (int a = 0; a < NA; ++a) acc[b][a] += fmaf(rb, Fx[a], fmaf(sb, gx[a], tb * Fx[a]));
        }
        continue;
      }
      float* base = dE + (size_t)q * cells + (size_t)f.je * it.ncol + f.ie;
#pragma unroll
      for (int b = 0; b < NU; ++b) {
        const float rb = cw * Fy[b], sb = cx * Fy[b], tb = cy * gy[b];
#pragma unroll
        for (int a = 0; a < NU; ++a) {
          const float v = fmaf(rb, Fx[a], fmaf(sb, gx[a], tb * Fx[a]));
          if (v != 0.0f) atomicAdd(base + b * it.ncol + a, v);
        }
      }
    }
  }
  flush_acc<NA>(acc, acc_ie, acc_je, dE, it.ncol);
  cnt.reduce_into(cnt_dst);
  ordered_misses_into(it, cnt_dst);
  __syncthreads();
  RayCount::publish(s_cnt, it.stats);
}

// Derivative maps of a collimated lens of degrees (p, q), 1 <= p, q <= 5 (the
// Sec. 3.1 figure shows (5, 3) beside (3, 3)), filter sizes 1 to 11: each lane
// traces its run of cells with the basis functions of the ray's span computed
// by the recursion (no power-form tables), and adds
//   dE_ij += (dw F_ij + w (dF_ij/dX dX + dF_ij/dY dY)) / (w_x w_y)
// for every direction with global atomics, as k_tangent.
__global__ void __launch_bounds__(256) k_tangent_general(const __grid_constant__ Item it, int warps,
                                                         const float* __restrict__ dP, int n_dirs,
                                                         float* __restrict__ dE) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_P = reinterpret_cast<float*>(smem);   // the heights
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  const int nctrl = it.ncu * it.ncv;
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) s_P[q] = __ldg(it.ctrl + q);
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const size_t cells = (size_t)it.ncol * it.nrow;
  const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
  const float inv_nsu = 1.0f / (float)it.nsu, inv_nsv = 1.0f / (float)it.nsv;
  RayCount cnt{0u};
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  uint64_t a0, a1;
  lane_range(it, warps, &a0, &a1);
  for (uint64_t id = a0; id < a1; ++id) {
    const uint32_t row = (uint32_t)(id / (uint64_t)it.cols), col = (uint32_t)(id % (uint64_t)it.cols);
    float ja = 0.5f, jb = 0.5f;
    if (it.jitter) {
      const uint2 w = philox_ray_words(it.seed, id);
      ja = unit23(w.x);
      jb = unit23(w.y);
    }
    const float u = ((float)col + ja) * inv_cols, v = ((float)row + jb) * inv_rows;
    float Nu[6], dNu[6], Nv[6], dNv[6];
    int k, l;
    basis_general(it.p, it.nsu, u, &k, Nu, dNu);
    basis_general(it.q, it.nsv, v, &l, Nv, dNv);
    float Z, Zu, Zv;
    surface_general(s_P, it.ncv, k, l, it.p, it.q, Nu, dNu, Nv, dNv, &Z, &Zu, &Zv);
    RayFwd r;
    // slopes per unit of span coordinate s = u nsu - k, as the cubic kernels
    collimated_at(it, u, v, fmaf(2.0f, v, -1.0f) * it.ry, Z, Zu * inv_nsu, Zv * inv_nsv, r);
    cnt.add(r.status, cnt_dst);
    if (r.status != FR_RAY_ON_SCREEN) continue;
    FootDyn f;
    if (!footprint_dyn(it, r.X, r.Y, f)) continue;
    float Fx[kWideNu], Fy[kWideNu], gx[kWideNu], gy[kWideNu];
    filter_grad_dyn(it, f, Fx, Fy, gx, gy);
    const float K = r.w * it.inv_area;
#pragma unroll 1
    for (int q = 0; q < n_dirs; ++q) {
      float dZ, dZu, dZv;
      surface_general(dP + (size_t)q * nctrl, it.ncv, k, l, it.p, it.q, Nu, dNu, Nv, dNv, &dZ, &dZu, &dZv);
      const RayTan tg = ray_tangent<true>(it, r, 0.0f, 0.0f, dZ, dZu * inv_nsu, dZv * inv_nsv);
      const float cw = tg.dw * it.inv_area, cx = K * tg.dX, cy = K * tg.dY;
      float* base = dE + (size_t)q * cells + (size_t)f.je * it.ncol + f.ie;
#pragma unroll 1
      for (int b = 0; b < it.nu; ++b) {
        const float rb = cw * Fy[b], sb = cx * Fy[b], tb = cy * gy[b];
#pragma unroll 1
        for (int a = 0; a < it.nu; ++a) {
          const float val = fmaf(rb, Fx[a], fmaf(sb, gx[a], tb * Fx[a]));
          if (val != 0.0f) atomicAdd(base + b * it.ncol + a, val);
        }
      }
    }
  }
  cnt.reduce_into(cnt_dst);
  __syncthreads();
  RayCount::publish(s_cnt, it.stats);
}

using TanKernel = void (*)(Item, int, const float*, int, float*);

TanKernel pick_tangent(int nu) {
  switch (nu) {
    case 1: return k_tangent<1>;
    case 3: return k_tangent<3>;
    case 5: return k_tangent<5>;
    case 7: return k_tangent<7>;
    case 9: return k_tangent<9>;
    default: return k_tangent<11>;
  }
}

}  // namespace

size_t tan_general_smem_bytes(const Item& it) { return (size_t)it.ncu * it.ncv * sizeof(float); }

cudaError_t launch_tangent_general(const Item& it, int warps, int grid, const float* dP, int n_dirs, float* dE,
                                   cudaStream_t st) {
  k_tangent_general<<<grid, warps * 32, tan_general_smem_bytes(it), st>>>(it, warps, dP, n_dirs, dE);
  return cudaGetLastError();
}

size_t tan_smem_bytes(const Item& it) {
  return ((lens_smem_bytes(it.nsu, it.nsv, needs_hull(it)) + 15) & ~(size_t)15) + (size_t)it.nsu * it.nsv * 4;
}

cudaError_t launch_tangent(const Item& it, int warps, int grid, size_t smem, const float* dP, int n_dirs, float* dE,
                           cudaStream_t st) {
  pick_tangent(it.nu)<<<grid, warps * 32, smem, st>>>(it, warps, dP, n_dirs, dE);
  return cudaGetLastError();
}

int tangent_occupancy(int threads, size_t smem, int nu) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_tangent(nu), threads, smem);
  return n;
}

cudaError_t configure_tangent(int optin) {
  for (int nu = 1; nu <= 11; nu += 2) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, pick_tangent(nu));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(pick_tangent(nu), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)a.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fr
