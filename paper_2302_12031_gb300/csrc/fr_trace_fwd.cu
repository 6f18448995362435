// Forward trace kernel (rows a1-a7) and the per-ray debug kernel.
//
// Each CTA works on one lens (item). It first builds that lens's tables in
// shared memory (the power form of the B-spline on every knot span, the basis
// tables and the convex-hull bounds, Sec. 2.1), then every lane traces an equal
// run of consecutive ray ids (lane_range), so the CTA's rays come from one
// compact part of the aperture. For a collimated source without jitter the
// row cubics of the current patch are kept in registers along a grid row.
// Each lane keeps the nu x nu footprint of its last ray in registers and adds
// the next ray there while the footprint does not move; it flushes the
// registers (with atomics) when it does: consecutive collimated rays usually
// share a pixel, so most rays cost no atomic. The flush goes to a privatised
// histogram in shared memory when the extended grid fits, else straight to
// global memory. A point-source lens whose grid does not fit privatises a
// central window of it; flushes outside the window go to global memory as
// 16-byte vector reductions (one per aligned group of four cells).
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

// Where flushed footprints go. Float mode with a shared-memory histogram keeps
// it as unsigned 32-bit fixed point (integer shared atomics are native and
// twice as fast as float ones): sh_scale is a power of two chosen so that the
// CTA's rays cannot overflow a cell (each ray adds at most flux/(n w_x w_y) to
// a cell). Deterministic mode keeps int64 fixed point at the global scale.
struct Target {
  bool smem;
  int ncol;
  float sh_scale;
  unsigned int* sh_u;
  unsigned long long* sh_q;
  float* gl_f;
  unsigned long long* gl_q;
  // Window form (float mode): sh_u holds rows wr0..wr1-1, columns wc0..wc1-1
  // (wcol = wc1 - wc0 per row); vec: gl_f is 16-byte aligned.
  bool win, vec;
  int wr0, wr1, wc0, wc1, wcol, ncell;
};

// Adds NU consecutive values v to global cells idx..idx+NU-1, where
// OFF = idx mod 4: one float4 reduction per aligned group of four cells
// (zeros in the lanes outside the run); groups that would pass the end of the
// grid are added cell by cell.
template <int NU, int OFF>
__device__ __forceinline__ void red_run_vec(float* g, int idx, int ncell, const float (&v)[NU]) {
  constexpr int NCH = (OFF + NU + 3) / 4;
  const int c0 = idx - OFF;
#pragma unroll
  for (int m = 0; m < NCH; ++m) {
    const int c = c0 + 4 * m;
    float l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * m + j - OFF;
      l[j] = (k >= 0 && k < NU) ? v[k] : 0.0f;
    }
    if (c + 4 <= ncell) {
      atomicAdd(reinterpret_cast<float4*>(g + c), make_float4(l[0], l[1], l[2], l[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * m + j - OFF;
        if (k >= 0 && k < NU) atomicAdd(g + c + j, l[j]);
      }
    }
  }
}

template <int NU>
__device__ __forceinline__ void red_run(const Target& tg, int idx, const float (&v)[NU]) {
  if (!tg.vec) {
#pragma unroll
    for (int a = 0; a < NU; ++a) atomicAdd(tg.gl_f + idx + a, v[a]);
    return;
  }
  switch (idx & 3) {
    case 0: red_run_vec<NU, 0>(tg.gl_f, idx, tg.ncell, v); break;
    case 1: red_run_vec<NU, 1>(tg.gl_f, idx, tg.ncell, v); break;
    case 2: red_run_vec<NU, 2>(tg.gl_f, idx, tg.ncell, v); break;
    default: red_run_vec<NU, 3>(tg.gl_f, idx, tg.ncell, v); break;
  }
}

template <int NU, bool DET>
struct FootAcc {
  int ie, je;
  typename AccT<DET>::type v[NU][NU];
};

// WIN: the kernel may run in the window form (single point-source lens, float mode).
template <int NU, bool DET, bool WIN = false>
__device__ __forceinline__ void acc_flush(FootAcc<NU, DET>& acc, const Target& tg, Bbox& bb) {
  if (acc.ie < 0) return;
  bb.imin = min(bb.imin, acc.ie);
  bb.imax = max(bb.imax, acc.ie);
  bb.jmin = min(bb.jmin, acc.je);
  bb.jmax = max(bb.jmax, acc.je);
  const int base = acc.je * tg.ncol + acc.ie;
  if constexpr (WIN && !DET) {
    if (tg.win) {
      const bool cols_in = acc.ie >= tg.wc0 && acc.ie + NU <= tg.wc1;
#pragma unroll
      for (int b = 0; b < NU; ++b) {
        const int row = acc.je + b;
        if (cols_in && row >= tg.wr0 && row < tg.wr1) {
          unsigned int* sh = tg.sh_u + (row - tg.wr0) * tg.wcol + (acc.ie - tg.wc0);
#pragma unroll
          for (int a = 0; a < NU; ++a) atomicAdd(sh + a, __float2uint_rn(acc.v[b][a] * tg.sh_scale));
        } else {
          red_run<NU>(tg, base + b * tg.ncol, acc.v[b]);
        }
      }
      acc.ie = -1;
      return;
    }
  }
#pragma unroll
  for (int b = 0; b < NU; ++b) {
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      const auto val = acc.v[b][a];
      const int idx = base + b * tg.ncol + a;
      if constexpr (DET) {
        if (tg.smem) atomicAdd(tg.sh_q + idx, (unsigned long long)val);
        else atomicAdd(tg.gl_q + idx, (unsigned long long)val);
      } else {
        if (tg.smem) atomicAdd(tg.sh_u + idx, __float2uint_rn(val * tg.sh_scale));
        else atomicAdd(tg.gl_f + idx, val);
      }
    }
  }
  acc.ie = -1;
}

// E_ij += w F_ij / (w_x w_y), F_ij = (f_i / S_x) (f_j / S_y).
template <int NU, bool DET, bool WIN = false>
__device__ __forceinline__ void deposit(const Item& it, const RayFwd& r, const Target& tg, FootAcc<NU, DET>& acc,
                                        Bbox& bb) {
  Foot<NU> f;
  if (!footprint<NU>(it, r.X, r.Y, f)) return;
  if (f.ie != acc.ie || f.je != acc.je) {
    acc_flush<NU, DET, WIN>(acc, tg, bb);
    acc.ie = f.ie;
    acc.je = f.je;
#pragma unroll
    for (int b = 0; b < NU; ++b)
#pragma unroll
      for (int a = 0; a < NU; ++a) acc.v[b][a] = 0;
  }
  // kx_a = w/(w_x w_y) F^x_a, ky_b = F^y_b, as packed pairs
  const float2 K = make_float2(r.w * it.inv_area * f.rsx, f.rsy);
  float kx[NU], ky[NU];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    const float2 k2 = __fmul2_rn(make_float2(f.fx[a], f.fy[a]), K);
    kx[a] = k2.x;
    ky[a] = k2.y;
  }
#pragma unroll
  for (int b = 0; b < NU; ++b) {
    if constexpr (DET) {
#pragma unroll
      for (int a = 0; a < NU; ++a) acc.v[b][a] += __float2ll_rn(kx[a] * ky[b] * it.fixE);
    } else {
      // acc_ba += kx_a ky_b, two cells of the row per instruction
#pragma unroll
      for (int a = 0; a + 1 < NU; a += 2) {
        const float2 s2 = __ffma2_rn(make_float2(kx[a], kx[a + 1]), make_float2(ky[b], ky[b]),
                                     make_float2(acc.v[b][a], acc.v[b][a + 1]));
        acc.v[b][a] = s2.x;
        acc.v[b][a + 1] = s2.y;
      }
      if (NU & 1) acc.v[b][NU - 1] = fmaf(kx[NU - 1], ky[b], acc.v[b][NU - 1]);
    }
  }
}

// KINDS: bit 0 = the kernel handles collimated items, bit 1 = point-source items.
// KINDS bit 2: the kernel also handles two-face lenses (entry tables in li).
// KINDS bit 3: point-source intersections march in the kernel (no deferred pass).
template <int NU, bool DET, int KINDS>
__device__ void run_lane(const Item& it, const LensSmem& ls, const LensSmem& li, const Target& tg, uint64_t a,
                         uint64_t b, float zmin, float zmax, RayCount& cnt, unsigned int* s_cnt, Bbox& bb,
                         unsigned int* s_group) {
  constexpr bool MARCH = (KINDS & 8) != 0;
  // Kernels that take point-source items may run the window form (float mode).
  constexpr bool WINK = (KINDS & 2) != 0;
  FootAcc<NU, DET> acc;
  acc.ie = -1;
  if constexpr ((KINDS & 4) != 0) {
    if (it.two_face) {
      // ray ids [a, b), or with a ray order chunks dealt to neighbouring lanes
      OrderCursor oc;
      if (it.order) oc.init(it, false);
      uint64_t next_id = a;
      for (;;) {
        uint64_t id;
        if (it.order) {
          if (!oc.valid()) break;
          id = __ldg(it.order + oc.p);
          oc.advance();
        } else {
          if (next_id >= b) break;
          id = next_id++;
        }
        RayFwd r;
        RayIn e;
        const uint32_t row = it.kind == FR_SOURCE_COLLIMATED ? (uint32_t)(id / (uint64_t)it.cols) : 0u;
        const uint32_t col = it.kind == FR_SOURCE_COLLIMATED ? (uint32_t)(id % (uint64_t)it.cols) : 0u;
        trace_two_face(it, ls, li, id, row, col, r, e);
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, WINK>(it, r, tg, acc, bb);
      }
      acc_flush<NU, DET, WINK>(acc, tg, bb);
      return;
    }
  }
  if ((KINDS & 2) && it.order) {
    // Ray order: groups of 32 neighbouring chunks, CTA c of the item owning
    // groups c, c + ctas, c + 2 ctas, ... and its warps taking them one at a
    // time from a shared counter (the cost of a group varies with the region
    // of the lens it covers; a fixed dealing leaves warps waiting on the
    // slowest); lane L of a warp walks chunk L of its group. The next id is
    // loaded one ray ahead, its latency hidden behind the current ray's trace.
    const uint64_t H = ordered_hits(it);
    const uint64_t ctas = (uint64_t)(it.cta_end - it.cta_begin), cta = (uint64_t)((int)blockIdx.x - it.cta_begin);
    const uint64_t lane = threadIdx.x & 31;
    for (;;) {
      __syncwarp();
      unsigned int k = 0u;
      if (lane == 0) k = atomicAdd(s_group, 1u);
      const uint64_t c0 = (cta + (uint64_t)__shfl_sync(0xffffffffu, k, 0) * ctas) * 32;
      if (c0 * kOrderChunk >= H) break;
      const uint64_t p0 = (c0 + lane) * kOrderChunk, hi = min(p0 + kOrderChunk, H);
      uint32_t next = p0 < hi ? __ldg(it.order + p0) : 0u;
      for (uint64_t p = p0; p < hi; ++p) {
        const uint64_t id = next;
        if (p + 1 < hi) next = __ldg(it.order + p + 1);
        RayFwd r;
        trace_point<MARCH>(it, ls, id, zmin, zmax, r);
        if (!MARCH && r.status == kRayDeferred) {
          defer_ray(it, id);
          continue;
        }
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, WINK>(it, r, tg, acc, bb);
      }
    }
  } else if ((KINDS & 1) && ((KINDS & 2) == 0 || it.kind == FR_SOURCE_COLLIMATED) && !it.jitter) {
    // cell centres in column lockstep (the lanes' shares are not lane_range's)
    const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
    Lockstep lk;
    lk.init(it, blockDim.x >> 5);
    uint32_t row, col, j0, j1;
    while (lk.next(it, &row, &col, &j0, &j1)) {
      RowWalk w;
      w.begin(it, ls, row, col, inv_cols, inv_rows);
      for (uint32_t j = j0; j < j1; ++j) {
        RayFwd r;
        w.trace(it, ls, j, r);
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, WINK>(it, r, tg, acc, bb);
      }
    }
  } else if (a < b) {
    if ((KINDS & 1) && ((KINDS & 2) == 0 || it.kind == FR_SOURCE_COLLIMATED)) {
      // jittered rays: the lane's run of ids
      const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
      uint32_t row = (uint32_t)(a / (uint64_t)it.cols);
      uint32_t col = (uint32_t)(a - (uint64_t)row * (uint64_t)it.cols);
      const uint32_t n = (uint32_t)(b - a);
      for (uint32_t j = 0; j < n; ++j) {
        RayFwd r;
        trace_collimated(it, ls, row, col, a + j, inv_cols, inv_rows, r);
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, WINK>(it, r, tg, acc, bb);
        if (++col == (uint32_t)it.cols) { col = 0; ++row; }
      }
    } else if (KINDS & 2) {
      for (uint64_t id = a; id < b; ++id) {
        RayFwd r;
        trace_point<MARCH>(it, ls, id, zmin, zmax, r);
        if (!MARCH && r.status == kRayDeferred) {
          defer_ray(it, id);
          continue;
        }
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, WINK>(it, r, tg, acc, bb);
      }
    }
  }
  acc_flush<NU, DET, WINK>(acc, tg, bb);
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Launch bounds: two CTAs per SM of up to 384 (collimated: float with filter
// sizes 1, 3 and 5, deterministic with 1 and 3), 256 (collimated deterministic
// with 5; batches); the single point-source
// kernel also runs one CTA per SM of 640 threads (filter sizes 1, 3) or 512
// (size 5) in the window form. The variants of filter sizes 1 and 3 do not
// spill; those of size 5 spill 150-200 bytes at any two-CTA bound.
template <int CAP, bool DET, int NU, int KINDS>
__global__ void __launch_bounds__(KINDS == 1 ? (NU <= 3 ? 384 : (DET ? 256 : 384))
                                             : ((KINDS & 7) == 2 ? (!DET && NU <= 3 ? 640 : 512) : 256),
                                  (KINDS & 7) == 2 ? 1 : 2)
    k_forward(const __grid_constant__ Launch<CAP> L) {
  pdl_trigger();   // the loss kernel may start launching; it waits for this one to end
  // One lens: item 0 by a constant index (its fields are then operands of the
  // parameter bank, not loads); a batch: the item whose CTA range holds this CTA.
  int ii = 0;
  if constexpr (CAP > 1)
    while (ii + 1 < L.n_items && (int)blockIdx.x >= L.items[ii].cta_end) ++ii;
  const Item& it = L.items[CAP > 1 ? ii : 0];
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = carve_exit(smem, it);
  const LensSmem li = (KINDS & 4) && it.two_face ? carve_entry(smem, it) : ls;
  unsigned char* hist_raw = smem + tables_bytes(it);
  const int ncell = it.ncol * it.nrow;
  uint64_t a, b;
  lane_range(it, L.warps, &a, &b);
  Target tg;
  tg.smem = it.smem_hist == 1;
  tg.ncol = it.ncol;
  tg.sh_u = reinterpret_cast<unsigned int*>(hist_raw);
  tg.sh_q = reinterpret_cast<unsigned long long*>(hist_raw);
  tg.gl_f = it.E;
  tg.gl_q = it.Efix;
  tg.win = !DET && it.smem_hist == 2;
  tg.vec = (reinterpret_cast<uintptr_t>(it.E) & 15) == 0;
  tg.wr0 = it.win_r0;
  tg.wr1 = it.win_r1;
  tg.wc0 = it.win_c0;
  tg.wc1 = it.win_c1;
  tg.wcol = it.win_c1 - it.win_c0;
  tg.ncell = ncell;
  {
    // 2^31 / (rays of this CTA x largest contribution of one ray), a power of two.
    const uint64_t n = it.ray_end - it.ray_begin;
    const uint64_t G = (uint64_t)(it.cta_end - it.cta_begin);
    const uint64_t ci = (uint64_t)((int)blockIdx.x - it.cta_begin);
    const bool lockstep = it.kind == FR_SOURCE_COLLIMATED && !it.jitter && !((KINDS & 4) && it.two_face);
    const float rays = (float)((KINDS & 2) && it.order ? OrderCursor::max_per_cta(it, L.warps)
                               : lockstep ? Lockstep::max_per_cta(it, L.warps)
                                          : n * (ci + 1) / G - n * ci / G) + 1.0f;
    int e = 0;
    frexpf(rays * it.omega0 * it.inv_area, &e);
    tg.sh_scale = ldexpf(1.0f, 31 - e);
  }
  if (tg.smem) {
    if constexpr (DET) {
      for (int q = threadIdx.x; q < ncell; q += blockDim.x) tg.sh_q[q] = 0ull;
    } else {
      for (int q = threadIdx.x; q < ncell; q += blockDim.x) tg.sh_u[q] = 0u;
    }
  } else if (tg.win) {
    const int nwin = (tg.wr1 - tg.wr0) * tg.wcol;
    for (int q = threadIdx.x; q < nwin; q += blockDim.x) tg.sh_u[q] = 0u;
  }
  __shared__ int s_bb[4];
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  __shared__ unsigned int s_group;
  if (threadIdx.x < 4) s_bb[threadIdx.x] = (threadIdx.x & 1) ? -1 : 0x7fffffff;
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  if (threadIdx.x == 0) s_group = 0u;
  if ((KINDS & 4) && it.two_face) build_two_face_tables(it, ls, li);   // ends with __syncthreads
  else build_lens_tables(it, ls);
  float zmin = 0.0f, zmax = 0.0f;
  if (it.kind == FR_SOURCE_POINT) zbounds(ls, &zmin, &zmax);
  RayCount cnt;
  cnt.on_screen = 0u;
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  Bbox bb{0x7fffffff, -1, 0x7fffffff, -1};
  // Launched early (programmatic launch, the previous kernel clears E): wait
  // for it before the first write to global memory, which with a shared
  // histogram is the final flush, else the first deposit.
  if (!tg.smem) pdl_wait();
  run_lane<NU, DET, KINDS>(it, ls, li, tg, a, b, zmin, zmax, cnt, cnt_dst, bb, &s_group);
  cnt.reduce_into(cnt_dst);
  ordered_misses_into(it, cnt_dst);
  if (tg.smem) pdl_wait();
  if (tg.smem || tg.win) {
    // Touched window: warp reductions, then one shared atomic per warp.
    const int i0 = __reduce_min_sync(0xffffffffu, bb.imin), i1 = __reduce_max_sync(0xffffffffu, bb.imax);
    const int j0 = __reduce_min_sync(0xffffffffu, bb.jmin), j1 = __reduce_max_sync(0xffffffffu, bb.jmax);
    if ((threadIdx.x & 31) == 0 && i1 >= 0) {
      atomicMin(&s_bb[0], i0);
      atomicMax(&s_bb[1], i1);
      atomicMin(&s_bb[2], j0);
      atomicMax(&s_bb[3], j1);
    }
  }
  __syncthreads();
  if (tg.smem && s_bb[1] >= 0) {
    // Flush the touched window of the privatised histogram.
    const int c0 = s_bb[0], c1 = s_bb[1] + NU - 1, r0 = s_bb[2], r1 = s_bb[3] + NU - 1;
    const int wcols = c1 - c0 + 1, n = wcols * (r1 - r0 + 1);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int rr = r0 + q / wcols, cc = c0 + q % wcols;
      const int idx = rr * it.ncol + cc;
      if constexpr (DET) {
        const unsigned long long v = tg.sh_q[idx];
        if (v) atomicAdd(tg.gl_q + idx, v);
      } else {
        const unsigned int v = tg.sh_u[idx];
        if (v) atomicAdd(tg.gl_f + idx, (float)v / tg.sh_scale);
      }
    }
  }
  if constexpr ((KINDS & 2) != 0 && !DET) {
    if (tg.win && s_bb[1] >= 0) {
      // Flush the touched part of the window: per row, one float4 reduction
      // per aligned group of four global cells.
      const int r0 = max(tg.wr0, s_bb[2]), r1 = min(tg.wr1 - 1, s_bb[3] + NU - 1);
      const int c0 = max(tg.wc0, s_bb[0]), c1 = min(tg.wc1 - 1, s_bb[1] + NU - 1);
      const float inv_scale = 1.0f / tg.sh_scale;
      const int maxch = (c1 - c0 + 3) / 4 + 1;          // groups a run of c1 - c0 + 1 cells can touch
      const int n = r0 <= r1 && c0 <= c1 ? (r1 - r0 + 1) * maxch : 0;
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int rr = r0 + q / maxch, m = q % maxch;
        const int gA = rr * tg.ncol + c0, gB = rr * tg.ncol + c1;
        const int c = (gA & ~3) + 4 * m;
        if (c > gB) continue;
        const unsigned int* srow = tg.sh_u + (rr - tg.wr0) * tg.wcol;
        float l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int g = c + j;
          l[j] = (g >= gA && g <= gB) ? (float)srow[g - rr * tg.ncol - tg.wc0] * inv_scale : 0.0f;
        }
        if (tg.vec && c + 4 <= ncell) {
          if (l[0] != 0.0f || l[1] != 0.0f || l[2] != 0.0f || l[3] != 0.0f)
            atomicAdd(reinterpret_cast<float4*>(tg.gl_f + c), make_float4(l[0], l[1], l[2], l[3]));
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (l[j] != 0.0f) atomicAdd(tg.gl_f + c + j, l[j]);
        }
      }
    }
  }
  RayCount::publish(s_cnt, it.stats);
}

// The deferred pass of the forward trace: the rays of each item's deferred
// list (hot kernel rays whose intersection needs the march) traced again with
// the march, one ray per thread, deposited straight into global memory (float
// atomics into E, or int64 into the fixed-point accumulator); their statuses
// are counted here. The last CTA resets the lists' counters for the next call.
template <int CAP, bool DET, int NU>
__global__ void __launch_bounds__(256) k_forward_deferred(const __grid_constant__ Launch<CAP> L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  for (int ii = 0; ii < L.n_items; ++ii) {
    const Item& it = L.items[ii];
    if (!it.defer) continue;
    const uint32_t n = *(volatile const uint32_t*)it.defer_n;
    if (n == 0) continue;
    const LensSmem ls = carve_exit(smem, it);
    if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
    build_lens_tables(it, ls);   // ends with __syncthreads
    float zmin, zmax;
    zbounds(ls, &zmin, &zmax);
    Target tg;
    tg.smem = false;
    tg.win = false;
    tg.vec = false;
    tg.ncol = it.ncol;
    tg.gl_f = it.E;
    tg.gl_q = it.Efix;
    Bbox bb{0x7fffffff, -1, 0x7fffffff, -1};
    RayCount cnt;
    cnt.on_screen = 0u;
    unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
    FootAcc<NU, DET> acc;
    acc.ie = -1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      RayFwd r;
      trace_point<true>(it, ls, it.ray_begin + it.defer[i], zmin, zmax, r);
      cnt.add(r.status, cnt_dst);
      if (r.status == FR_RAY_ON_SCREEN) deposit<NU, DET, false>(it, r, tg, acc, bb);
    }
    acc_flush<NU, DET, false>(acc, tg, bb);
    cnt.reduce_into(cnt_dst);
    __syncthreads();
    RayCount::publish(s_cnt, it.stats);
    __syncthreads();   // the tables of the next item reuse the shared memory
  }
  // every CTA has read the counters: the last one resets them
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(L.items[0].defer_n + 1, 1u);
    s_last = done + 1 == gridDim.x;
  }
  __syncthreads();
  if (s_last && threadIdx.x < (unsigned int)L.n_items) {
    const Item& it = L.items[threadIdx.x];
    if (it.defer) *it.defer_n = 0u;
    if (threadIdx.x == 0) L.items[0].defer_n[1] = 0u;
  }
}

// The full record of every ray of [ray_begin, ray_end), one thread per ray.
// Forward trace for filter sizes 7, 9 and 11 (one single-face lens per
// launch, the size a runtime value) and, GEN, for a collimated lens of other
// degrees (any filter size): each lane traces its run of rays (of ordered
// positions for a point source in the ray order), point sources with the
// march in the kernel, GEN lenses by the basis recursion on the heights in
// shared memory, and adds every ray's nu x nu footprint straight to the
// privatised histogram (float or, deterministic, int64 fixed point) when the
// grid fits in shared memory, else to global memory. The per-ray terms are
// those of `deposit`: kx_a ky_b with kx_a = w/(w_x w_y) f_a / S_x and
// ky_b = f_b / S_y.
template <bool DET, bool GEN>
__global__ void __launch_bounds__(256) k_forward_wide(const __grid_constant__ Launch<1> L) {
  pdl_wait();   // launched early after a kernel that triggers: nothing before it ends
  const Item& it = L.items[0];
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = GEN ? LensSmem{} : carve_exit(smem, it);
  float* sP = reinterpret_cast<float*>(smem);
  const bool sh = it.smem_hist == 1;
  float* sh_f = reinterpret_cast<float*>(smem + tables_bytes(it));
  unsigned long long* sh_q = reinterpret_cast<unsigned long long*>(smem + tables_bytes(it));
  const int ncell = it.ncol * it.nrow;
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  __shared__ int s_bb[4];
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  if (threadIdx.x < 4) s_bb[threadIdx.x] = (threadIdx.x & 1) ? -1 : 0x7fffffff;
  if (sh)
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
      if constexpr (DET) sh_q[q] = 0ull;
      else sh_f[q] = 0.0f;
    }
  if constexpr (GEN) {
    for (int q = threadIdx.x; q < it.ncu * it.ncv; q += blockDim.x) sP[q] = __ldg(it.ctrl + q);
    __syncthreads();
  } else {
    build_lens_tables(it, ls);   // ends with __syncthreads
  }
  float zmin = 0.0f, zmax = 0.0f;
  if (!GEN && it.kind == FR_SOURCE_POINT) zbounds(ls, &zmin, &zmax);
  const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
  uint64_t a, b;
  lane_range(it, L.warps, &a, &b);
  RayCount cnt;
  cnt.on_screen = 0u;
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  Bbox bb{0x7fffffff, -1, 0x7fffffff, -1};
  for (uint64_t p = a; p < b; ++p) {
    RayFwd r;
    if constexpr (GEN) {
      int k, l;
      float Nu[6], dNu[6], Nv[6], dNv[6];
      trace_collimated_general(it, sP, p, inv_cols, inv_rows, r, &k, &l, Nu, dNu, Nv, dNv);
    } else if (it.kind == FR_SOURCE_COLLIMATED) {
      const uint32_t row = (uint32_t)(p / (uint64_t)it.cols), col = (uint32_t)(p % (uint64_t)it.cols);
      trace_collimated(it, ls, row, col, p, inv_cols, inv_rows, r);
    } else {
      trace_point<true>(it, ls, it.order ? (uint64_t)__ldg(it.order + p) : p, zmin, zmax, r);
    }
    cnt.add(r.status, cnt_dst);
    if (r.status != FR_RAY_ON_SCREEN) continue;
    FootDyn f;
    if (!footprint_dyn(it, r.X, r.Y, f)) continue;
    bb.imin = min(bb.imin, f.ie);
    bb.imax = max(bb.imax, f.ie);
    bb.jmin = min(bb.jmin, f.je);
    bb.jmax = max(bb.jmax, f.je);
    const float Kx = r.w * it.inv_area * f.rsx;
#pragma unroll 1
    for (int rb = 0; rb < it.nu; ++rb) {
      const float ky = f.fy[rb] * f.rsy;
      if (ky == 0.0f) continue;
      const int row0 = (f.je + rb) * it.ncol + f.ie;
#pragma unroll 1
      for (int ca = 0; ca < it.nu; ++ca) {
        const float kx = f.fx[ca] * Kx;
        if (kx == 0.0f) continue;
        if constexpr (DET) {
          const unsigned long long v = (unsigned long long)__float2ll_rn(kx * ky * it.fixE);
          if (sh) atomicAdd(sh_q + row0 + ca, v);
          else atomicAdd(it.Efix + row0 + ca, v);
        } else {
          if (sh) atomicAdd(sh_f + row0 + ca, kx * ky);
          else atomicAdd(it.E + row0 + ca, kx * ky);
        }
      }
    }
  }
  cnt.reduce_into(cnt_dst);
  ordered_misses_into(it, cnt_dst);
  if (sh) {
    const int i0 = __reduce_min_sync(0xffffffffu, bb.imin), i1 = __reduce_max_sync(0xffffffffu, bb.imax);
    const int j0 = __reduce_min_sync(0xffffffffu, bb.jmin), j1 = __reduce_max_sync(0xffffffffu, bb.jmax);
    if ((threadIdx.x & 31) == 0 && i1 >= 0) {
      atomicMin(&s_bb[0], i0);
      atomicMax(&s_bb[1], i1);
      atomicMin(&s_bb[2], j0);
      atomicMax(&s_bb[3], j1);
    }
  }
  __syncthreads();
  if (sh && s_bb[1] >= 0) {
    // the touched window of the privatised histogram
    const int c0 = s_bb[0], c1 = s_bb[1] + it.nu - 1, r0 = s_bb[2], r1 = s_bb[3] + it.nu - 1;
    const int wcols = c1 - c0 + 1, n = wcols * (r1 - r0 + 1);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int idx = (r0 + q / wcols) * it.ncol + c0 + q % wcols;
      if constexpr (DET) {
        const unsigned long long v = sh_q[idx];
        if (v) atomicAdd(it.Efix + idx, v);
      } else {
        const float v = sh_f[idx];
        if (v != 0.0f) atomicAdd(it.E + idx, v);
      }
    }
  }
  RayCount::publish(s_cnt, it.stats);
}

__global__ void __launch_bounds__(128) k_debug(const __grid_constant__ Item it, fr_ray_record* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = carve_exit(smem, it);
  const LensSmem li = it.two_face ? carve_entry(smem, it) : ls;
  if (it.two_face) build_two_face_tables(it, ls, li);
  else build_lens_tables(it, ls);
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t id = it.ray_begin + i;
  if (id >= it.ray_end) return;
  RayFwd r;
  r.status = FR_RAY_ON_SCREEN;
  r.k = r.l = -1;
  r.u = r.v = r.s = r.t = r.x = r.y = r.z = r.dx = r.dy = r.dz = 0.0f;
  r.tx = r.ty = r.tz = r.w = r.X = r.Y = r.tstar = 0.0f;
  r.iters = 0;
  if (it.two_face) {
    RayIn e;
    const uint32_t row = it.kind == FR_SOURCE_COLLIMATED ? (uint32_t)(id / (uint64_t)it.cols) : 0u;
    const uint32_t col = it.kind == FR_SOURCE_COLLIMATED ? (uint32_t)(id % (uint64_t)it.cols) : 0u;
    trace_two_face(it, ls, li, id, row, col, r, e);
  } else if (it.kind == FR_SOURCE_COLLIMATED) {
    const uint32_t row = (uint32_t)(id / (uint64_t)it.cols), col = (uint32_t)(id % (uint64_t)it.cols);
    trace_collimated(it, ls, row, col, id, 1.0f / (float)it.cols, 1.0f / (float)it.rows, r);
  } else {
    float zmin, zmax;
    zbounds(ls, &zmin, &zmax);
    trace_point<true>(it, ls, id, zmin, zmax, r);
  }
  fr_ray_record rec;
  rec.status = r.status;
  rec.span_i = r.k >= 0 ? r.k + 3 : -1;
  rec.span_j = r.l >= 0 ? r.l + 3 : -1;
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
  size_t b = tables_bytes(it);
  if (it.smem_hist == 2) b += (size_t)(it.win_r1 - it.win_r0) * (it.win_c1 - it.win_c0) * 4;
  else if (it.smem_hist) b += (size_t)it.ncol * it.nrow * (det ? 8 : 4);
  return b;
}

size_t lens_tables_bytes(const Item& it) { return tables_bytes(it); }

// The kernel variant for (deterministic, nu, kinds); KINDS as in run_lane.
template <int CAP>
using FwdKernel = void (*)(Launch<CAP>);

template <int CAP, bool DET, int KINDS>
FwdKernel<CAP> pick_nu(int nu) {
  return nu == 1 ? k_forward<CAP, DET, 1, KINDS> : (nu == 3 ? k_forward<CAP, DET, 3, KINDS> : k_forward<CAP, DET, 5, KINDS>);
}

template <int CAP>
FwdKernel<CAP> pick_forward(bool det, int nu, int kinds);
template <>
FwdKernel<1> pick_forward<1>(bool det, int nu, int kinds) {
  if (nu > 5) return det ? k_forward_wide<true, false> : k_forward_wide<false, false>;   // filter sizes 7, 9, 11
  if (kinds == 1) return det ? pick_nu<1, true, 1>(nu) : pick_nu<1, false, 1>(nu);
  if (kinds == 4) return det ? pick_nu<1, true, 7>(nu) : pick_nu<1, false, 7>(nu);   // two-face lens
  if (kinds == 8) return det ? pick_nu<1, true, 10>(nu) : pick_nu<1, false, 10>(nu);  // point, march in the kernel
  return det ? pick_nu<1, true, 2>(nu) : pick_nu<1, false, 2>(nu);
}
template <>
FwdKernel<kMaxItems> pick_forward<kMaxItems>(bool det, int nu, int) {
  return det ? pick_nu<kMaxItems, true, 3>(nu) : pick_nu<kMaxItems, false, 3>(nu);
}

template <int CAP>
cudaError_t launch_forward(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st, bool pdl,
                           bool march) {
  const int threads = 32 * L.warps;
  if constexpr (CAP == 1) {
    if (L.items[0].p != 3 || L.items[0].q != 3)   // a collimated lens of other degrees
      return launch_k(det ? k_forward_wide<true, true> : k_forward_wide<false, true>, dim3(grid), dim3(threads),
                      smem, st, pdl, L);
  }
  int kinds = L.items[0].two_face ? 4 : (L.items[0].kind == FR_SOURCE_COLLIMATED ? 1 : 2);
  if (march && kinds == 2) kinds = 8;
  return launch_k(pick_forward<CAP>(det, L.items[0].nu, kinds), dim3(grid), dim3(threads), smem, st, pdl, L);
}
template cudaError_t launch_forward<1>(const Launch<1>&, int, size_t, bool, cudaStream_t, bool, bool);
template cudaError_t launch_forward<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t, bool, bool);

template <int CAP>
using FwdDeferredKernel = void (*)(Launch<CAP>);

template <int CAP>
FwdDeferredKernel<CAP> pick_forward_deferred(bool det, int nu) {
  if (det) return nu == 1 ? k_forward_deferred<CAP, true, 1> : (nu == 3 ? k_forward_deferred<CAP, true, 3>
                                                                          : k_forward_deferred<CAP, true, 5>);
  return nu == 1 ? k_forward_deferred<CAP, false, 1> : (nu == 3 ? k_forward_deferred<CAP, false, 3>
                                                                 : k_forward_deferred<CAP, false, 5>);
}

template <int CAP>
cudaError_t launch_forward_deferred(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st) {
  return launch_k(pick_forward_deferred<CAP>(det, L.items[0].nu), dim3(grid), dim3(256), smem, st, false, L);
}
template cudaError_t launch_forward_deferred<1>(const Launch<1>&, int, size_t, bool, cudaStream_t);
template cudaError_t launch_forward_deferred<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t);

cudaError_t launch_debug(const Item& it, fr_ray_record* out, cudaStream_t st) {
  const uint64_t n = it.ray_end - it.ray_begin;
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  const unsigned int blocks = (unsigned int)((n + threads - 1) / threads);
  k_debug<<<blocks, threads, tables_bytes(it), st>>>(it, out);
  return cudaGetLastError();
}

int forward_occupancy(int threads, size_t smem, bool det, bool batch, int nu, int kinds) {
  int n = 0;
  if (batch) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_forward<kMaxItems>(det, nu, kinds), threads, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_forward<1>(det, nu, kinds), threads, smem);
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
  if ((e = allow_max_smem(k_debug, optin))) return e;
  for (int det = 0; det < 2; ++det)
    for (int nu = 1; nu <= 5; nu += 2) {
      for (int kinds = 1; kinds <= 8; kinds *= 2)
        if ((e = allow_max_smem(pick_forward<1>(det != 0, nu, kinds), optin))) return e;
      if ((e = allow_max_smem(pick_forward<kMaxItems>(det != 0, nu, 3), optin))) return e;
      if ((e = allow_max_smem(pick_forward_deferred<1>(det != 0, nu), optin))) return e;
      if ((e = allow_max_smem(pick_forward_deferred<kMaxItems>(det != 0, nu), optin))) return e;
    }
  if ((e = allow_max_smem(k_forward_wide<false, false>, optin))) return e;
  if ((e = allow_max_smem(k_forward_wide<true, false>, optin))) return e;
  if ((e = allow_max_smem(k_forward_wide<false, true>, optin))) return e;
  if ((e = allow_max_smem(k_forward_wide<true, true>, optin))) return e;
  return cudaSuccess;
}

}  // namespace fr
