// Adjoint kernel (row a9): reverse mode of the forward trace, recomputing each
// ray's path from its id instead of storing it.
//
// The CTA builds its lens's tables in shared memory as the forward kernel does
// and every lane takes the same run of rays. Per ray: the forward code of
// fr_device.cuh runs again; dL/dE is gathered on the nu x nu footprint (kept in
// registers while the footprint does not move); ray_reverse() carries it back
// through the filter, propagation, Schlick, Snell and the normal (and, for
// point sources, the intersection by the implicit function theorem) to three
// adjoints (zeta, Zs_bar, Zt_bar); the 16 control-point gradients of the ray's
// knot span are
//   dL/dP_{k+a,l+b} += zeta N_a N_b + Zs_bar N'_a N_b + Zt_bar N_a N'_b,
// summed in registers while the span does not change, then flushed to a
// CTA-private copy of dL/dP in shared memory that is added to global memory
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

// Float mode, called by all 32 lanes of a converged warp: the register sums of
// the lanes that hold sums of the same patch as the first lane with sums are
// added up by a reduce-scatter over the warp (16 shuffle rounds, after which
// lane 2j holds the total of term j), one shared atomic per control point; the
// other lanes flush their own.
__device__ __forceinline__ void grad_flush_warp(GradAcc<false>& acc, int ncv, float* sg) {
  const unsigned int full = 0xffffffffu;
  const unsigned int key = acc.k >= 0 ? (((unsigned int)acc.k << 16) | (unsigned int)acc.l) : full;
  const unsigned int with_sums = __ballot_sync(full, key != full);
  if (with_sums == 0u) return;
  const unsigned int key0 = __shfl_sync(full, key, __ffs(with_sums) - 1);
  const int k0 = (int)(key0 >> 16), l0 = (int)(key0 & 0xffffu);
  const unsigned int lane = threadIdx.x & 31u;
  const bool mine = key == key0;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {   // first exchange: halves of the 16 terms over lane bit 4
    const bool hi = (lane & 16u) != 0;
    const float lo_t = mine ? acc.g[i >> 2][i & 3] : 0.0f;
    const float hi_t = mine ? acc.g[(i + 8) >> 2][(i + 8) & 3] : 0.0f;
    v[i] = (hi ? hi_t : lo_t) + __shfl_xor_sync(full, hi ? lo_t : hi_t, 16);
  }
#pragma unroll
  for (int w = 4, bit = 8; w >= 1; w >>= 1, bit >>= 1) {
    const bool hi = (lane & (unsigned int)bit) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) v[i] = (hi ? v[i + w] : v[i]) + __shfl_xor_sync(full, hi ? v[i] : v[i + w], bit);
  }
  const float tot = v[0] + __shfl_xor_sync(full, v[0], 1);
  const int term = (int)(lane >> 1);   // lane bits 4..1 picked the term's bits 3..0
  if ((lane & 1u) == 0u && tot != 0.0f) atomicAdd(sg + (k0 + (term >> 2)) * ncv + l0 + (term & 3), tot);
  if (!mine) grad_flush<false>(acc, ncv, sg, nullptr);
  acc.k = -1;
}

struct GradOut {
  float* sg_f;
  unsigned long long* sg_q;
  float fixP;
  unsigned int* s_group;   // the CTA's next group of ordered chunks (shared memory)
};

// The footprint of dL/dE, re-read only when the footprint moves.
template <int NU>
struct GCache {
  int ie, je;
  float G[NU][NU];
};

// dL/dP += zeta N_a N_b + Zs_bar N'_a N_b + Zt_bar N_a N'_b for a ray on
// patch (k, l) (N_b, N'_b at the ray's t in Nv, dNv), summed in `acc` while the
// patch does not change; on the triangle mesh the height term follows the
// triangle's vertices.
template <bool DET, bool COLL>
__device__ __forceinline__ void add_ray_grad(const Item& it, const LensSmem& ls, const RayFwd& r, float zeta,
                                             float Zsb, float Ztb, const float (&Nv)[4], const float (&dNv)[4],
                                             GradAcc<DET>& acc, const GradOut& go) {
  float Nu[4], dNu[4];
  basis_eval(ls.bu + r.k * 4, r.s, Nu, dNu);
  if (r.k != acc.k || r.l != acc.l) {
    grad_flush<DET>(acc, it.ncv, go.sg_f, go.sg_q);
    acc.k = r.k;
    acc.l = r.l;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc.g[a][b] = 0;
  }
  if (!COLL && it.mesh_nu > 0) {
    // Triangle mesh: the hit height follows the triangle's vertices, the
    // normal the B-spline at the hit.
    float W[4][4];
    int kt, lt;
    mesh_vertex_weights(it, ls, r, W, &kt, &lt);
    const bool same = kt == r.k && lt == r.l;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float A = Zsb * dNu[a], B = Ztb * Nu[a];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float c = fmaf(same ? zeta : 0.0f, W[a][b], fmaf(A, Nv[b], B * dNv[b]));
        if constexpr (DET) acc.g[a][b] += __float2ll_rn(c * go.fixP);
        else acc.g[a][b] += c;
      }
    }
    if (!same) {   // rare: the triangle lies in the neighbouring patch
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float c = zeta * W[a][b];
          const int idx = (kt + a) * it.ncv + lt + b;
          if constexpr (DET) atomicAdd(go.sg_q + idx, (unsigned long long)__float2ll_rn(c * go.fixP));
          else atomicAdd(go.sg_f + idx, c);
        }
    }
    return;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float A = fmaf(zeta, Nu[a], Zsb * dNu[a]);
    const float B = Ztb * Nu[a];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float c = fmaf(A, Nv[b], B * dNv[b]);
      if constexpr (DET) acc.g[a][b] += __float2ll_rn(c * go.fixP);
      else acc.g[a][b] += c;
    }
  }
}

template <int NU, bool DET, bool COLL>
__device__ __forceinline__ void adjoint_ray(const Item& it, const LensSmem& ls, const RayFwd& r, GCache<NU>& gc,
                                            const float (&Nv)[4], const float (&dNv)[4], GradAcc<DET>& acc,
                                            const GradOut& go) {
  Foot<NU> f;
  if (!footprint_scalar<NU>(it, r.X, r.Y, f)) return;
  if (f.ie != gc.ie || f.je != gc.je) {
#pragma unroll
    for (int b = 0; b < NU; ++b)
#pragma unroll
      for (int a = 0; a < NU; ++a) gc.G[b][a] = __ldg(it.dLdE + (size_t)(f.je + b) * it.ncol + f.ie + a);
    gc.ie = f.ie;
    gc.je = f.je;
  }
  float zeta, Zsb, Ztb;
  ray_reverse<NU, COLL>(it, ls, r, f, gc.G, &zeta, &Zsb, &Ztb);
  add_ray_grad<DET, COLL>(it, ls, r, zeta, Zsb, Ztb, Nv, dNv, acc, go);
}

// Along one grid row of a collimated source t, N_b(t) and N'_b(t) are fixed, so
// the 16 gradient terms of the rays that fall in one patch factor through
// power moments of s:
//   sum_rays (zeta N_a(s) + Zs_bar N'_a(s)) = sum_e c_ae M_e + sum_e e c_ae D_{e-1},
//   sum_rays Zt_bar N_a(s) = sum_e c_ae Q_e,
// with N_a(s) = sum_e c_ae s^e, M_e = sum zeta s^e, D_e = sum Zs_bar s^e,
// Q_e = sum Zt_bar s^e. The moments are summed per ray and expanded through the
// basis table only when the patch or the row changes (float mode).
struct RowMoments {
  int k, l;
  uint32_t row;
  float M0, M1, M2, M3, D0, D1, D2, Q0, Q1, Q2, Q3;
};

__device__ __forceinline__ void moments_flush(RowMoments& m, const LensSmem& ls, int ncv, const float (&Nv)[4],
                                              const float (&dNv)[4], float* sg) {
  if (m.k < 0) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float4 c = ls.bu[m.k * 4 + a];
    const float SA = fmaf(c.x, m.M0, fmaf(c.y, m.M1, fmaf(c.z, m.M2, fmaf(c.w, m.M3,
                     fmaf(c.y, m.D0, fmaf(2.0f * c.z, m.D1, 3.0f * c.w * m.D2))))));
    const float SB = fmaf(c.x, m.Q0, fmaf(c.y, m.Q1, fmaf(c.z, m.Q2, c.w * m.Q3)));
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float v = fmaf(SA, Nv[b], SB * dNv[b]);
      if (v != 0.0f) atomicAdd(sg + (m.k + a) * ncv + m.l + b, v);
    }
  }
  m.k = -1;
}

template <int NU>
__device__ __forceinline__ void adjoint_ray_moments(const Item& it, const LensSmem& ls, const RayFwd& r,
                                                    uint32_t row, GCache<NU>& gc, RowMoments& m,
                                                    const float (&Nv)[4], const float (&dNv)[4], float* sg) {
  Foot<NU> f;
  if (!footprint_scalar<NU>(it, r.X, r.Y, f)) return;
  if (f.ie != gc.ie || f.je != gc.je) {
#pragma unroll
    for (int b = 0; b < NU; ++b)
#pragma unroll
      for (int a = 0; a < NU; ++a) gc.G[b][a] = __ldg(it.dLdE + (size_t)(f.je + b) * it.ncol + f.ie + a);
    gc.ie = f.ie;
    gc.je = f.je;
  }
  float zeta, Zsb, Ztb;
  ray_reverse<NU, true>(it, ls, r, f, gc.G, &zeta, &Zsb, &Ztb);
  if (r.k != m.k || row != m.row) {
    moments_flush(m, ls, it.ncv, Nv, dNv, sg);
    m.k = r.k;
    m.l = r.l;
    m.row = row;
    m.M0 = m.M1 = m.M2 = m.M3 = m.D0 = m.D1 = m.D2 = m.Q0 = m.Q1 = m.Q2 = m.Q3 = 0.0f;
  }
  const float s = r.s, s2 = s * s, s3 = s2 * s;
  // the same sums as packed pairs (each lane rounds as the scalar operation)
  const float2 zd = make_float2(zeta, Zsb);
  float2 v = __fadd2_rn(make_float2(m.M0, m.D0), zd);
  m.M0 = v.x;
  m.D0 = v.y;
  v = __ffma2_rn(zd, make_float2(s, s), make_float2(m.M1, m.D1));
  m.M1 = v.x;
  m.D1 = v.y;
  v = __ffma2_rn(zd, make_float2(s2, s2), make_float2(m.M2, m.D2));
  m.M2 = v.x;
  m.D2 = v.y;
  v = __ffma2_rn(make_float2(zeta, Ztb), make_float2(s3, s3), make_float2(m.M3, m.Q3));
  m.M3 = v.x;
  m.Q3 = v.y;
  v = __ffma2_rn(make_float2(Ztb, Ztb), make_float2(s, s2), make_float2(m.Q1, m.Q2));
  m.Q1 = v.x;
  m.Q2 = v.y;
  m.Q0 += Ztb;
}

// dL/dP_{k+a,l+b} += zeta N_a N_b + Zs_bar N'_a N_b + Zt_bar N_a N'_b at (s, t)
// of patch (k, l) of a net whose tables are `tab`, summed in `acc`.
template <bool DET>
__device__ __forceinline__ void grad_add(const LensSmem& tab, int k, int l, float s, float t, float zeta, float Zsb,
                                         float Ztb, int ncv, GradAcc<DET>& acc, float* sg_f,
                                         unsigned long long* sg_q, float fixP) {
  float Nu[4], dNu[4], Nv[4], dNv[4];
  basis_eval(tab.bu + k * 4, s, Nu, dNu);
  basis_eval(tab.bv + l * 4, t, Nv, dNv);
  if (k != acc.k || l != acc.l) {
    grad_flush<DET>(acc, ncv, sg_f, sg_q);
    acc.k = k;
    acc.l = l;
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

// Two-face lens: both nets' gradients; the entry net's follow the exit net's
// in dL/dP.
template <int NU, bool DET>
__device__ void run_adjoint_lane_two(const Item& it, const LensSmem& ls, const LensSmem& li, uint64_t a, uint64_t b,
                                     const GradOut& go, RayCount& cnt, unsigned int* s_cnt) {
  GradAcc<DET> acc, acc_in;
  acc.k = acc_in.k = -1;
  GCache<NU> gc;
  gc.ie = gc.je = -1;
  const int nout = it.ncu * it.ncv;
  float* sgi_f = go.sg_f + nout;
  unsigned long long* sgi_q = go.sg_q + nout;
  // ray ids [a, b), or with a ray order chunks dealt far apart (OrderCursor)
  OrderCursor oc;
  if (it.order) oc.init(it, true);
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
    if (r.status != FR_RAY_ON_SCREEN) continue;
    Foot<NU> f;
    if (!footprint_scalar<NU>(it, r.X, r.Y, f)) continue;
    if (f.ie != gc.ie || f.je != gc.je) {
#pragma unroll
      for (int bb = 0; bb < NU; ++bb)
#pragma unroll
        for (int aa = 0; aa < NU; ++aa) gc.G[bb][aa] = __ldg(it.dLdE + (size_t)(f.je + bb) * it.ncol + f.ie + aa);
      gc.ie = f.ie;
      gc.je = f.je;
    }
    float z, zs, zt, zi, zsi, zti;
    ray_reverse_two<NU>(it, ls, li, r, e, f, gc.G, &z, &zs, &zt, &zi, &zsi, &zti);
    grad_add<DET>(ls, r.k, r.l, r.s, r.t, z, zs, zt, it.ncv, acc, go.sg_f, go.sg_q, go.fixP);
    grad_add<DET>(li, e.k, e.l, e.s, e.t, zi, zsi, zti, it.ncv_in, acc_in, sgi_f, sgi_q, go.fixP);
  }
  grad_flush<DET>(acc, it.ncv, go.sg_f, go.sg_q);
  grad_flush<DET>(acc_in, it.ncv_in, sgi_f, sgi_q);
}

// KINDS: bit 0 = the kernel handles collimated items, bit 1 = point-source
// items, bit 2 = two-face lenses (entry tables in li).
template <int NU, bool DET, int KINDS>
__device__ void run_adjoint_lane(const Item& it, const LensSmem& ls, const LensSmem& li, uint64_t a, uint64_t b,
                                 float zmin, float zmax, const GradOut& go, RayCount& cnt, unsigned int* s_cnt) {
  if constexpr ((KINDS & 4) != 0) {
    if (it.two_face) {
      run_adjoint_lane_two<NU, DET>(it, ls, li, a, b, go, cnt, s_cnt);
      return;
    }
  }
  GradAcc<DET> acc;
  acc.k = -1;
  GCache<NU> gc;
  gc.ie = gc.je = -1;
  if ((KINDS & 2) && it.order && !DET) {
    // Ray order, float mode: groups of 32 neighbouring chunks, CTA c of the
    // item owning groups c, c + ctas, c + 2 ctas, ... and its warps taking
    // them one at a time from a shared counter (the cost of a group varies
    // with the region of the lens it covers; a fixed dealing leaves warps
    // waiting on the slowest). The lanes walk their chunks of the group in
    // step and the warp's sums are flushed together at the group's end. Next
    // id loaded one ray ahead.
    float Nv[4], dNv[4];
    const uint64_t H = ordered_hits(it);
    const uint64_t ctas = (uint64_t)(it.cta_end - it.cta_begin), cta = (uint64_t)((int)blockIdx.x - it.cta_begin);
    const uint64_t lane = threadIdx.x & 31;
    for (;;) {
      unsigned int k = 0u;
      if (lane == 0) k = atomicAdd(go.s_group, 1u);
      const uint64_t c0 = (cta + (uint64_t)__shfl_sync(0xffffffffu, k, 0) * ctas) * 32;
      if (c0 * kOrderChunk >= H) break;
      const uint64_t p0 = (c0 + lane) * kOrderChunk, hi = min(p0 + kOrderChunk, H);
      uint32_t next = p0 < hi ? __ldg(it.order + p0) : 0u;
      for (uint64_t p = p0; p < hi; ++p) {
        const uint64_t id = next;
        if (p + 1 < hi) next = __ldg(it.order + p + 1);
        RayFwd r;
        trace_point<false>(it, ls, id, zmin, zmax, r);
        if (r.status == kRayDeferred) {
          defer_ray(it, id);
          continue;
        }
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) {
          basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
          adjoint_ray<NU, DET, false>(it, ls, r, gc, Nv, dNv, acc, go);
        }
      }
      __syncwarp();
      if constexpr (!DET) grad_flush_warp(acc, it.ncv, go.sg_f);
    }
  } else if ((KINDS & 2) && it.order) {
    // Ray order, fixed point: chunks dealt far apart over the lanes
    // (OrderCursor), next id loaded one ray ahead.
    float Nv[4], dNv[4];
    OrderCursor oc;
    oc.init(it, true);
    uint32_t next = oc.valid() ? __ldg(it.order + oc.p) : 0u;
    while (oc.valid()) {
      const uint64_t id = next;
      oc.advance();
      if (oc.valid()) next = __ldg(it.order + oc.p);
      RayFwd r;
      trace_point<false>(it, ls, id, zmin, zmax, r);
      if (r.status == kRayDeferred) {
        defer_ray(it, id);
        continue;
      }
      cnt.add(r.status, s_cnt);
      if (r.status == FR_RAY_ON_SCREEN) {
        basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
        adjoint_ray<NU, DET, false>(it, ls, r, gc, Nv, dNv, acc, go);
      }
    }
  } else if (a < b) {
    if ((KINDS & 1) && ((KINDS & 2) == 0 || it.kind == FR_SOURCE_COLLIMATED)) {
      const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
      uint32_t row = (uint32_t)(a / (uint64_t)it.cols);
      uint32_t col = (uint32_t)(a - (uint64_t)row * (uint64_t)it.cols);
      float Nv[4], dNv[4];
      const uint32_t n = (uint32_t)(b - a);
      if (!it.jitter && !DET) {
        RowPatch rp;
        rp.row = 0xffffffffu;
        RowMoments m;
        m.k = -1;
        m.row = 0xffffffffu;
        uint32_t nv_row = 0xffffffffu;
        for (uint32_t j = 0; j < n; ++j) {
          RayFwd r;
          trace_collimated_row(it, ls, row, col, inv_cols, inv_rows, rp, r);
          cnt.add(r.status, s_cnt);
          if (r.status == FR_RAY_ON_SCREEN) {
            if (row != nv_row) {   // the v basis is fixed along a row
              moments_flush(m, ls, it.ncv, Nv, dNv, go.sg_f);   // moments of the previous row
              basis_eval(ls.bv + rp.l * 4, rp.t, Nv, dNv);
              nv_row = row;
            }
            adjoint_ray_moments<NU>(it, ls, r, row, gc, m, Nv, dNv, go.sg_f);
          }
          if (++col == (uint32_t)it.cols) { col = 0; ++row; }
        }
        moments_flush(m, ls, it.ncv, Nv, dNv, go.sg_f);
      } else if (!it.jitter) {
        RowPatch rp;
        rp.row = 0xffffffffu;
        uint32_t nv_row = 0xffffffffu;
        for (uint32_t j = 0; j < n; ++j) {
          RayFwd r;
          trace_collimated_row(it, ls, row, col, inv_cols, inv_rows, rp, r);
          cnt.add(r.status, s_cnt);
          if (r.status == FR_RAY_ON_SCREEN) {
            if (row != nv_row) {   // the v basis is fixed along a row
              basis_eval(ls.bv + rp.l * 4, rp.t, Nv, dNv);
              nv_row = row;
            }
            adjoint_ray<NU, DET, true>(it, ls, r, gc, Nv, dNv, acc, go);
          }
          if (++col == (uint32_t)it.cols) { col = 0; ++row; }
        }
      } else {
        for (uint32_t j = 0; j < n; ++j) {
          RayFwd r;
          trace_collimated(it, ls, row, col, a + j, inv_cols, inv_rows, r);
          cnt.add(r.status, s_cnt);
          if (r.status == FR_RAY_ON_SCREEN) {
            basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
            adjoint_ray<NU, DET, true>(it, ls, r, gc, Nv, dNv, acc, go);
          }
          if (++col == (uint32_t)it.cols) { col = 0; ++row; }
        }
      }
    } else if (KINDS & 2) {
      float Nv[4], dNv[4];
      for (uint64_t id = a; id < b; ++id) {
        RayFwd r;
        trace_point<false>(it, ls, id, zmin, zmax, r);
        if (r.status == kRayDeferred) {
          defer_ray(it, id);
          continue;
        }
        cnt.add(r.status, s_cnt);
        if (r.status == FR_RAY_ON_SCREEN) {
          basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
          adjoint_ray<NU, DET, false>(it, ls, r, gc, Nv, dNv, acc, go);
        }
      }
    }
  }
  grad_flush<DET>(acc, it.ncv, go.sg_f, go.sg_q);
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Launch bounds: two CTAs per SM of 320 threads for the single-lens collimated
// float kernel with filter sizes 1 and 3 (96 registers, no spills), 256 else.
template <int CAP, bool DET, int NU, int KINDS>
__global__ void __launch_bounds__(CAP == 1 && !DET && KINDS == 1 && NU <= 3 ? 320 : 256, 2)
    k_adjoint(const __grid_constant__ Launch<CAP> L) {
  // One lens: item 0 by a constant index (its fields are then operands of the
  // parameter bank, not loads); a batch: the item whose CTA range holds this CTA.
  int ii = 0;
  if constexpr (CAP > 1)
    while (ii + 1 < L.n_items && (int)blockIdx.x >= L.items[ii].cta_end) ++ii;
  const Item& it = L.items[CAP > 1 ? ii : 0];
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = carve_exit(smem, it);
  const LensSmem li = (KINDS & 4) && it.two_face ? carve_entry(smem, it) : ls;
  unsigned char* grad_raw = smem + tables_bytes(it);
  __shared__ unsigned int s_group;
  GradOut go;
  go.s_group = &s_group;
  go.sg_f = reinterpret_cast<float*>(grad_raw);
  go.sg_q = reinterpret_cast<unsigned long long*>(grad_raw);
  const int nctrl = it.nparam;
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) go.sg_q[q] = 0ull;
    else go.sg_f[q] = 0.0f;
  }
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  if (threadIdx.x == 0) s_group = 0u;
  pdl_trigger();
  // Launched to overlap the previous kernel: dL/dE only after it ends; the
  // lens too unless the caller has said that kernel does not write it.
  if (!L.early_lens) pdl_wait();
  if ((KINDS & 4) && it.two_face) build_two_face_tables(it, ls, li);   // ends with __syncthreads
  else build_lens_tables(it, ls);
  if (L.early_lens) pdl_wait();
  go.fixP = 0.0f;
  if constexpr (DET) {
    // Fixed-point scale 2^40 / (max|dL/dE| * flux / pixel area), a power of two.
    const float unit = *it.gmax * it.fixP_unit;
    int e = 0;
    if (unit > 0.0f) frexpf(unit, &e);
    go.fixP = unit > 0.0f ? ldexpf(1.0f, 40 - e) : 1.0f;
  }
  float zmin = 0.0f, zmax = 0.0f;
  if (it.kind == FR_SOURCE_POINT) zbounds(ls, &zmin, &zmax);
  uint64_t a, b;
  lane_range(it, L.warps, &a, &b);
  RayCount cnt;
  cnt.on_screen = 0u;
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  run_adjoint_lane<NU, DET, KINDS>(it, ls, li, a, b, zmin, zmax, go, cnt, cnt_dst);
  cnt.reduce_into(cnt_dst);
  ordered_misses_into(it, cnt_dst);
  __syncthreads();
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) {
      const unsigned long long v = go.sg_q[q];
      if (v) atomicAdd(it.Pfix + q, v);
    } else {
      const float v = go.sg_f[q];
      if (v != 0.0f) atomicAdd(it.dLdP + q, v);
    }
  }
  RayCount::publish(s_cnt, it.stats);
}

// The deferred pass of the adjoint: each item's deferred rays traced again
// with the march, one ray per thread, reversed, and their dL/dP terms added
// straight into global memory (the float gradient or the int64 accumulator at
// the adjoint kernel's scale); statuses counted here; the last CTA resets the
// lists' counters.
template <int CAP, bool DET, int NU>
__global__ void __launch_bounds__(256) k_adjoint_deferred(const __grid_constant__ Launch<CAP> L) {
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
    GradOut go;
    go.sg_f = it.dLdP;
    go.sg_q = it.Pfix;
    go.s_group = nullptr;
    go.fixP = 0.0f;
    if constexpr (DET) {   // the scale of k_adjoint
      const float unit = *it.gmax * it.fixP_unit;
      int e = 0;
      if (unit > 0.0f) frexpf(unit, &e);
      go.fixP = unit > 0.0f ? ldexpf(1.0f, 40 - e) : 1.0f;
    }
    RayCount cnt;
    cnt.on_screen = 0u;
    unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
    GradAcc<DET> acc;
    acc.k = -1;
    GCache<NU> gc;
    gc.ie = gc.je = -1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      RayFwd r;
      trace_point<true>(it, ls, it.ray_begin + it.defer[i], zmin, zmax, r);
      cnt.add(r.status, cnt_dst);
      if (r.status == FR_RAY_ON_SCREEN) {
        float Nv[4], dNv[4];
        basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
        adjoint_ray<NU, DET, false>(it, ls, r, gc, Nv, dNv, acc, go);
      }
    }
    grad_flush<DET>(acc, it.ncv, go.sg_f, go.sg_q);
    cnt.reduce_into(cnt_dst);
    __syncthreads();
    RayCount::publish(s_cnt, it.stats);
    __syncthreads();   // the tables of the next item reuse the shared memory
  }
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

// Deterministic mode: int64 fixed point -> float gradient, with the scale the
// adjoint kernel used (recomputed from the same device value).
// Adjoint for filter sizes 7, 9 and 11 (one single-face lens per launch, the
// size a runtime value) and, GEN, for a collimated lens of other degrees (any
// filter size): each lane traces its run of rays (of ordered positions for a
// point source in the ray order), point sources with the march in the
// kernel, GEN lenses by the basis recursion on the heights in shared memory;
// per ray the footprint's dL/dE is read from global memory inside the
// contraction (W = sum G F_x F_y, Xs = sum G F'_x F_y, Ys = sum G F_x F'_y),
// ray_reverse_tail gives the adjoints of the hit, and add_ray_grad sums the 16
// terms as in the other kernels (GEN: the (p+1)(q+1) terms
// zeta N_a N_b + Zs_bar dN_a/ds N_b + Zt_bar N_a dN_b/dt go to the CTA's copy
// of dL/dP ray by ray).
template <bool DET, bool GEN>
__global__ void __launch_bounds__(256) k_adjoint_wide(const __grid_constant__ Launch<1> L) {
  pdl_wait();   // launched early after a kernel that triggers: nothing before it ends
  const Item& it = L.items[0];
  extern __shared__ __align__(16) unsigned char smem[];
  const LensSmem ls = GEN ? LensSmem{} : carve_exit(smem, it);
  float* sP = reinterpret_cast<float*>(smem);
  unsigned char* grad_raw = smem + tables_bytes(it);
  GradOut go;
  go.s_group = nullptr;
  go.sg_f = reinterpret_cast<float*>(grad_raw);
  go.sg_q = reinterpret_cast<unsigned long long*>(grad_raw);
  const int nctrl = it.nparam;
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) go.sg_q[q] = 0ull;
    else go.sg_f[q] = 0.0f;
  }
  __shared__ unsigned int s_cnt[FR_RAY_NCAUSES];
  if (threadIdx.x < FR_RAY_NCAUSES) s_cnt[threadIdx.x] = 0u;
  if constexpr (GEN) {
    for (int q = threadIdx.x; q < it.ncu * it.ncv; q += blockDim.x) sP[q] = __ldg(it.ctrl + q);
    __syncthreads();
  } else {
    build_lens_tables(it, ls);   // ends with __syncthreads
  }
  go.fixP = 0.0f;
  if constexpr (DET) {   // the scale of k_adjoint
    const float unit = *it.gmax * it.fixP_unit;
    int e = 0;
    if (unit > 0.0f) frexpf(unit, &e);
    go.fixP = unit > 0.0f ? ldexpf(1.0f, 40 - e) : 1.0f;
  }
  float zmin = 0.0f, zmax = 0.0f;
  const bool coll = it.kind == FR_SOURCE_COLLIMATED;
  if (!GEN && !coll) zbounds(ls, &zmin, &zmax);
  const float inv_cols = 1.0f / (float)it.cols, inv_rows = 1.0f / (float)it.rows;
  uint64_t a, b;
  lane_range(it, L.warps, &a, &b);
  RayCount cnt;
  cnt.on_screen = 0u;
  unsigned int* cnt_dst = it.stats ? s_cnt : nullptr;
  GradAcc<DET> acc;
  acc.k = -1;
  for (uint64_t p = a; p < b; ++p) {
    RayFwd r;
    int gk = 0, gl = 0;
    float gNu[6], gdNu[6], gNv[6], gdNv[6];
    if constexpr (GEN) {
      trace_collimated_general(it, sP, p, inv_cols, inv_rows, r, &gk, &gl, gNu, gdNu, gNv, gdNv);
    } else if (coll) {
      const uint32_t row = (uint32_t)(p / (uint64_t)it.cols), col = (uint32_t)(p % (uint64_t)it.cols);
      trace_collimated(it, ls, row, col, p, inv_cols, inv_rows, r);
    } else {
      trace_point<true>(it, ls, it.order ? (uint64_t)__ldg(it.order + p) : p, zmin, zmax, r);
    }
    cnt.add(r.status, cnt_dst);
    if (r.status != FR_RAY_ON_SCREEN) continue;
    FootDyn f;
    if (!footprint_dyn(it, r.X, r.Y, f)) continue;
    float Fx[kWideNu], Fy[kWideNu], gxa[kWideNu], gya[kWideNu];
    filter_grad_dyn(it, f, Fx, Fy, gxa, gya);
    float W = 0.0f, Xs = 0.0f, Ys = 0.0f;
#pragma unroll 1
    for (int ca = 0; ca < it.nu; ++ca) {
      float A = 0.0f, B = 0.0f;
      const float* col = it.dLdE + (size_t)f.je * it.ncol + f.ie + ca;
#pragma unroll 1
      for (int rb = 0; rb < it.nu; ++rb) {
        const float g = __ldg(col + (size_t)rb * it.ncol);
        A = fmaf(g, Fy[rb], A);
        B = fmaf(g, gya[rb], B);
      }
      W = fmaf(A, Fx[ca], W);
      Xs = fmaf(A, gxa[ca], Xs);
      Ys = fmaf(B, Fx[ca], Ys);
    }
    float zeta, Zsb, Ztb, Nv[4], dNv[4];
    if constexpr (GEN) {
      ray_reverse_tail<true>(it, ls, r, W, Xs, Ys, &zeta, &Zsb, &Ztb);
      const float isu = 1.0f / (float)it.nsu, isv = 1.0f / (float)it.nsv;
#pragma unroll 1
      for (int ca = 0; ca <= it.p; ++ca) {
        const float A = fmaf(zeta, gNu[ca], Zsb * gdNu[ca] * isu), B = Ztb * gNu[ca] * isv;
#pragma unroll 1
        for (int cb = 0; cb <= it.q; ++cb) {
          const float c = fmaf(A, gNv[cb], B * gdNv[cb]);
          const int idx = (gk + ca) * it.ncv + gl + cb;
          if constexpr (DET) atomicAdd(go.sg_q + idx, (unsigned long long)__float2ll_rn(c * go.fixP));
          else if (c != 0.0f) atomicAdd(go.sg_f + idx, c);
        }
      }
      continue;
    }
    basis_eval(ls.bv + r.l * 4, r.t, Nv, dNv);
    if (coll) {
      ray_reverse_tail<true>(it, ls, r, W, Xs, Ys, &zeta, &Zsb, &Ztb);
      add_ray_grad<DET, true>(it, ls, r, zeta, Zsb, Ztb, Nv, dNv, acc, go);
    } else {
      ray_reverse_tail<false>(it, ls, r, W, Xs, Ys, &zeta, &Zsb, &Ztb);
      add_ray_grad<DET, false>(it, ls, r, zeta, Zsb, Ztb, Nv, dNv, acc, go);
    }
  }
  grad_flush<DET>(acc, it.ncv, go.sg_f, go.sg_q);
  cnt.reduce_into(cnt_dst);
  ordered_misses_into(it, cnt_dst);
  __syncthreads();
  for (int q = threadIdx.x; q < nctrl; q += blockDim.x) {
    if constexpr (DET) {
      const unsigned long long v = go.sg_q[q];
      if (v) atomicAdd(it.Pfix + q, v);
    } else {
      const float v = go.sg_f[q];
      if (v != 0.0f) atomicAdd(it.dLdP + q, v);
    }
  }
  RayCount::publish(s_cnt, it.stats);
}

__global__ void k_grad_fix_to_float(const __grid_constant__ Item it, int accumulate) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= it.nparam) return;
  const float unit = *it.gmax * it.fixP_unit;
  int e = 0;
  if (unit > 0.0f) frexpf(unit, &e);
  const double inv = unit > 0.0f ? ldexp(1.0, e - 40) : 1.0;
  const float v = (float)((double)(long long)it.Pfix[q] * inv);
  it.dLdP[q] = accumulate ? it.dLdP[q] + v : v;
}

}  // namespace

size_t adj_smem_bytes(const Item& it, bool det) {
  return tables_bytes(it) + (size_t)it.nparam * (det ? 8 : 4);
}

template <int CAP>
using AdjKernel = void (*)(Launch<CAP>);

template <int CAP, bool DET, int KINDS>
AdjKernel<CAP> pick_nu(int nu) {
  return nu == 1 ? k_adjoint<CAP, DET, 1, KINDS> : (nu == 3 ? k_adjoint<CAP, DET, 3, KINDS> : k_adjoint<CAP, DET, 5, KINDS>);
}

template <int CAP>
AdjKernel<CAP> pick_adjoint(bool det, int nu, int kinds);
template <>
AdjKernel<1> pick_adjoint<1>(bool det, int nu, int kinds) {
  if (nu > 5) return det ? k_adjoint_wide<true, false> : k_adjoint_wide<false, false>;   // filter sizes 7, 9, 11
  if (kinds == 1) return det ? pick_nu<1, true, 1>(nu) : pick_nu<1, false, 1>(nu);
  if (kinds == 4) return det ? pick_nu<1, true, 7>(nu) : pick_nu<1, false, 7>(nu);   // two-face lens
  return det ? pick_nu<1, true, 2>(nu) : pick_nu<1, false, 2>(nu);
}
template <>
AdjKernel<kMaxItems> pick_adjoint<kMaxItems>(bool det, int nu, int) {
  return det ? pick_nu<kMaxItems, true, 3>(nu) : pick_nu<kMaxItems, false, 3>(nu);
}

template <int CAP>
cudaError_t launch_adjoint(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st, bool pdl) {
  const int threads = 32 * L.warps;
  if constexpr (CAP == 1) {
    if (L.items[0].p != 3 || L.items[0].q != 3)   // a collimated lens of other degrees
      return launch_k(det ? k_adjoint_wide<true, true> : k_adjoint_wide<false, true>, dim3(grid), dim3(threads),
                      smem, st, pdl, L);
  }
  const int kinds = L.items[0].two_face ? 4 : (L.items[0].kind == FR_SOURCE_COLLIMATED ? 1 : 2);
  return launch_k(pick_adjoint<CAP>(det, L.items[0].nu, kinds), dim3(grid), dim3(threads), smem, st, pdl, L);
}
template cudaError_t launch_adjoint<1>(const Launch<1>&, int, size_t, bool, cudaStream_t, bool);
template cudaError_t launch_adjoint<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t, bool);

template <int CAP>
using AdjDeferredKernel = void (*)(Launch<CAP>);

template <int CAP>
AdjDeferredKernel<CAP> pick_adjoint_deferred(bool det, int nu) {
  if (det) return nu == 1 ? k_adjoint_deferred<CAP, true, 1> : (nu == 3 ? k_adjoint_deferred<CAP, true, 3>
                                                                          : k_adjoint_deferred<CAP, true, 5>);
  return nu == 1 ? k_adjoint_deferred<CAP, false, 1> : (nu == 3 ? k_adjoint_deferred<CAP, false, 3>
                                                                 : k_adjoint_deferred<CAP, false, 5>);
}

template <int CAP>
cudaError_t launch_adjoint_deferred(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st) {
  return launch_k(pick_adjoint_deferred<CAP>(det, L.items[0].nu), dim3(grid), dim3(256), smem, st, false, L);
}
template cudaError_t launch_adjoint_deferred<1>(const Launch<1>&, int, size_t, bool, cudaStream_t);
template cudaError_t launch_adjoint_deferred<kMaxItems>(const Launch<kMaxItems>&, int, size_t, bool, cudaStream_t);

cudaError_t launch_grad_fix_to_float(const Item& it, int accumulate, cudaStream_t st) {
  const int n = it.nparam;
  k_grad_fix_to_float<<<(n + 255) / 256, 256, 0, st>>>(it, accumulate);
  return cudaGetLastError();
}

int adjoint_occupancy(int threads, size_t smem, bool det, bool batch, int nu, int kinds) {
  int n = 0;
  if (batch) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_adjoint<kMaxItems>(det, nu, kinds), threads, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_adjoint<1>(det, nu, kinds), threads, smem);
  return n;
}

template <class K>
static cudaError_t allow_max_smem(K kernel, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}

cudaError_t configure_adjoint(int optin) {
  cudaError_t e;
  for (int det = 0; det < 2; ++det)
    for (int nu = 1; nu <= 5; nu += 2) {
      for (int kinds = 1; kinds <= 4; kinds *= 2)
        if ((e = allow_max_smem(pick_adjoint<1>(det != 0, nu, kinds), optin))) return e;
      if ((e = allow_max_smem(pick_adjoint<kMaxItems>(det != 0, nu, 3), optin))) return e;
      if ((e = allow_max_smem(pick_adjoint_deferred<1>(det != 0, nu), optin))) return e;
      if ((e = allow_max_smem(pick_adjoint_deferred<kMaxItems>(det != 0, nu), optin))) return e;
    }
  if ((e = allow_max_smem(k_adjoint_wide<false, false>, optin))) return e;
  if ((e = allow_max_smem(k_adjoint_wide<true, false>, optin))) return e;
  if ((e = allow_max_smem(k_adjoint_wide<false, true>, optin))) return e;
  if ((e = allow_max_smem(k_adjoint_wide<true, true>, optin))) return e;
  return cudaSuccess;
}

}  // namespace fr
