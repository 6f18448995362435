// Device functions of the freeform-lens trace: the lens tables each CTA builds
// in shared memory, counter-based ray generation, B-spline patch evaluation,
// refraction, propagation, the reconstruction filter and the reverse-mode
// derivatives of all of them.
#pragma once

#include <cstdint>

#include "fr_internal.h"

namespace fr {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (id_lo, id_hi,
// 0, 0), key = seed. Ten rounds of two 32x32->64-bit products; the key is bumped
// by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint2 philox_ray_words(uint64_t seed, uint64_t id) {
  uint32_t c0 = (uint32_t)id, c1 = (uint32_t)(id >> 32), c2 = 0u, c3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint2(c0, c1);
}

// Programmatic dependent launch: pdl_wait() returns once the kernel this one
// was launched to follow has completed and its writes are visible (at once
// when the launch did not ask for overlap); pdl_trigger() lets the next kernel
// on the stream begin launching before this one ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Top 23 bits of a word plus one half, times 2^-23: exact in FP32, in (0,1).
__device__ __forceinline__ float unit23(uint32_t w) {
  return fmaf((float)(w >> 9), 1.0f / 8388608.0f, 0.5f / 8388608.0f);
}

// PTX approximate instructions (single MUFU operations): 2^x with a relative
// error below 2^-22, 1/x within 1 ulp, sqrt below 2^-23 relative. All flush
// denormals to zero.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Square root with a relative error below 2^-23 (one MUFU operation).
__device__ __forceinline__ float fast_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// Sec. 2.1: the bicubic B-spline in power form. On knot span k of a clamped
// uniform knot vector with nspan spans, the four non-zero basis functions
// N_{k..k+3,3} are cubics in the local coordinate s = u*nspan - k; the
// Cox-de Boor recursion run on polynomials in s gives their coefficients. The
// knots are handled in units of the span width, where they are the integers
// K(j) = clamp(j-3, 0, nspan), so every ratio in the recursion is a ratio of
// small integers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int knot_units(int j, int nspan) { return min(max(j - 3, 0), nspan); }

__device__ inline void span_basis(int k, int nspan, float4 out[4]) {
  const int i = k + 3;  // knot index of the span's left end
  float poly[5][4];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) poly[a][e] = 0.0f;
  poly[3][0] = 1.0f;    // N_{i,0} = 1 on its own span
  const int Ki = knot_units(i, nspan);
#pragma unroll
  for (int d = 1; d <= 3; ++d) {
    float next[5][4];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) next[a][e] = 0.0f;
#pragma unroll
    for (int jj = 3 - d; jj <= 3; ++jj) {
      const int j = i - 3 + jj;
      // The denominators are knot differences of at most d <= 3 spans.
      const int den1 = knot_units(j + d, nspan) - knot_units(j, nspan);
      const int den2 = knot_units(j + d + 1, nspan) - knot_units(j + 1, nspan);
      const float r1 = den1 == 1 ? 1.0f : (den1 == 2 ? 0.5f : (den1 == 3 ? (1.0f / 3.0f) : 0.0f));
      const float r2 = den2 == 1 ? 1.0f : (den2 == 2 ? 0.5f : (den2 == 3 ? (1.0f / 3.0f) : 0.0f));
      // (u - u_j)/(u_{j+d} - u_j) = (Ki - K(j) + s)/den1
      const float a0 = (float)(Ki - knot_units(j, nspan)) * r1;
      const float a1 = r1;
      // (u_{j+d+1} - u)/(u_{j+d+1} - u_{j+1}) = (K(j+d+1) - Ki - s)/den2
      const float b0 = (float)(knot_units(j + d + 1, nspan) - Ki) * r2;
      const float b1 = -r2;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float c = a0 * poly[jj][e] + b0 * poly[jj + 1][e];
        if (e > 0) c += a1 * poly[jj][e - 1] + b1 * poly[jj + 1][e - 1];
        next[jj][e] = c;
      }
    }
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) poly[a][e] = next[a][e];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] = make_float4(poly[a][0], poly[a][1], poly[a][2], poly[a][3]);
}

// Tables of one lens in shared memory.
struct LensSmem {
  float4* patch;   // [nsu*nsv][4]: row e holds C[e][0..3] of Z = sum_{e,f} C[e][f] s^e t^f
  float4* bu;      // [nsu][4]: coefficients of N_{k+a}(s) in powers of s
  float4* bv;      // [nsv][4]
  int* zkey;       // [4]: min and max control height (convex hull, Sec. 2.1.2) as
                   // order-preserving integer keys, then the net's bounds on |Z_s|
                   // and |Z_t| as float bits (point sources only; see zbounds, slopes)
  float4* hull;    // [nsu*nsv] (nets that rays must intersect): per patch (zmin, zmax, Bs, Bt),
                   // see patch_hull
};

// Float <-> int key with the same order (for shared-memory atomicMin/Max).
__device__ __forceinline__ int float_key(float f) {
  const int b = __float_as_int(f);
  return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }

// The convex-hull bounds of the control heights (valid after build_lens_tables
// for point-source items).
__device__ __forceinline__ void zbounds(const LensSmem& s, float* zmin, float* zmax) {
  *zmin = key_float(s.zkey[0]);
  *zmax = key_float(s.zkey[1]);
}

// Bounds on |dZ/ds| and |dZ/dt| (patch coordinates) over the whole net (valid
// after build_net_tables for nets with hull tables).
__device__ __forceinline__ void slopes(const LensSmem& s, float* gs, float* gt) {
  *gs = __int_as_float(s.zkey[2]);
  *gt = __int_as_float(s.zkey[3]);
}

// Bytes of one net's tables; `hull`: with the per-patch bounds of the
// intersection (nets that rays must intersect: the exit net of a point source,
// both nets of a two-face lens).
__host__ __device__ inline size_t lens_smem_bytes(int nsu, int nsv, bool hull) {
  return (size_t)(nsu * nsv * (hull ? 5 : 4) + (nsu + nsv) * 4) * sizeof(float4) + 16;
}

// Whether an item's nets carry the intersection bounds.
__host__ __device__ inline bool needs_hull(const Item& it) { return it.kind == FR_SOURCE_POINT || it.two_face; }

// Bytes of all lens tables of an item (the exit net's, then the entry net's).
__host__ __device__ inline size_t tables_bytes(const Item& it) {
  // a lens of other degrees (collimated, general-degree kernels): its heights
  if (it.p != 3 || it.q != 3) return ((size_t)it.ncu * it.ncv * sizeof(float) + 15) & ~(size_t)15;
  const bool h = needs_hull(it);
  size_t b = (lens_smem_bytes(it.nsu, it.nsv, h) + 15) & ~(size_t)15;
  if (it.two_face) b += (lens_smem_bytes(it.nsu_in, it.nsv_in, h) + 15) & ~(size_t)15;
  return b;
}

__device__ inline LensSmem carve_lens(unsigned char* base, int nsu, int nsv, bool hull) {
  LensSmem s;
  s.patch = reinterpret_cast<float4*>(base);
  s.bu = s.patch + nsu * nsv * 4;
  s.bv = s.bu + nsu * 4;
  s.zkey = reinterpret_cast<int*>(s.bv + nsv * 4);
  s.hull = hull ? s.bv + nsv * 4 + 1 : nullptr;   // after the 16 bytes of zkey
  return s;
}

// Bounds of one bicubic patch for the intersection, from its own control net
// in the Bernstein (Bezier) basis, b_ij, obtained from the power form C[e][f]:
// along each direction b_i = sum_{e <= i} binom(i,e)/binom(3,e) c_e. By the
// convex-hull property of the Bernstein basis (the patch form of Sec. 2.1.2's
// argument) Z lies in [min b, max b] on the patch, and its second derivatives in
// patch coordinates are bounded by the hull of the differenced net:
//   |Z_ss| <= 6 max |b_{i+2,j} - 2 b_{i+1,j} + b_ij|, |Z_tt| likewise,
//   |Z_st| <= 9 max |b_{i+1,j+1} - b_{i+1,j} - b_{i,j+1} + b_ij|.
// Along a line (s, t) = (s0 + a tau, t0 + b tau) this gives
//   |d2Z/dtau2| <= Z_ss a^2 + 2 |Z_st| |a b| + Z_tt b^2 <= Bs a^2 + Bt b^2,
// Bs = Mss + Mst, Bt = Mtt + Mst (2|ab| <= a^2 + b^2). The bounds are widened
// a little for FP32 rounding. Returns (zmin, zmax, Bs, Bt); *ms, *mt bound
// |Z_s| and |Z_t| on the patch (3 times the largest first difference).
__device__ inline float4 patch_hull(const float (&C)[4][4], float* ms, float* mt) {
  float T[4][4], B[4][4];
  const float third = 1.0f / 3.0f;
#pragma unroll
  for (int f = 0; f < 4; ++f) {   // along s
    T[0][f] = C[0][f];
    T[1][f] = fmaf(third, C[1][f], C[0][f]);
    T[2][f] = fmaf(third, C[2][f], fmaf(2.0f * third, C[1][f], C[0][f]));
    T[3][f] = C[0][f] + C[1][f] + C[2][f] + C[3][f];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {   // along t
    B[i][0] = T[i][0];
    B[i][1] = fmaf(third, T[i][1], T[i][0]);
    B[i][2] = fmaf(third, T[i][2], fmaf(2.0f * third, T[i][1], T[i][0]));
    B[i][3] = T[i][0] + T[i][1] + T[i][2] + T[i][3];
  }
  float zmn = B[0][0], zmx = B[0][0], mss = 0.0f, mtt = 0.0f, mst = 0.0f, babs = 0.0f, m1s = 0.0f, m1t = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      zmn = fminf(zmn, B[i][j]);
      zmx = fmaxf(zmx, B[i][j]);
      babs = fmaxf(babs, fabsf(B[i][j]));
      if (i < 2) mss = fmaxf(mss, fabsf(B[i + 2][j] - 2.0f * B[i + 1][j] + B[i][j]));
      if (j < 2) mtt = fmaxf(mtt, fabsf(B[i][j + 2] - 2.0f * B[i][j + 1] + B[i][j]));
      if (i < 3 && j < 3) mst = fmaxf(mst, fabsf(B[i + 1][j + 1] - B[i + 1][j] - B[i][j + 1] + B[i][j]));
      if (i < 3) m1s = fmaxf(m1s, fabsf(B[i + 1][j] - B[i][j]));
      if (j < 3) m1t = fmaxf(m1t, fabsf(B[i][j + 1] - B[i][j]));
    }
  const float pad = 4e-6f * (1.0f + babs);   // rounding of the conversions above
  mss = fmaf(6.0f, mss, 24.0f * pad);
  mtt = fmaf(6.0f, mtt, 24.0f * pad);
  mst = fmaf(9.0f, mst, 36.0f * pad);
  *ms = fmaf(3.0f, m1s, 6.0f * pad);   // |Z_s| <= 3 max |b_{i+1,j} - b_ij|
  *mt = fmaf(3.0f, m1t, 6.0f * pad);
  return make_float4(zmn - pad, zmx + pad, mss + mst, mtt + mst);
}

// Every thread of the CTA takes part; ends with __syncthreads.
//   Z(s,t) = sum_{a,b} N_{k+a}(s) N_{l+b}(t) P^z_{k+a,l+b} = sum_{e,f} C[e][f] s^e t^f,
//   C[e][f] = sum_a sum_b Bu[a][e] Bv[b][f] P^z_{k+a,l+b}.
// For point sources the min and max control height come out of the same
// loads (every control point lies in some patch's 4x4 window).
__device__ inline void build_net_tables(const float* ctrl, int ncv, int nsu, int nsv, bool bounds,
                                        const LensSmem& s) {
  if (bounds && threadIdx.x == 0) {
    s.zkey[0] = 0x7fffffff;
    s.zkey[1] = (int)0x80000000;
    s.zkey[2] = 0;   // +0.0f
    s.zkey[3] = 0;
  }
  for (int q = threadIdx.x; q < nsu + nsv; q += blockDim.x) {
    const bool isu = q < nsu;
    const int k = isu ? q : q - nsu;
    float4 B[4];
    span_basis(k, isu ? nsu : nsv, B);
    float4* dst = (isu ? s.bu : s.bv) + k * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a) dst[a] = B[a];
  }
  __syncthreads();
  const int npatch = nsu * nsv;
  float zmn = INFINITY, zmx = -INFINITY, gs = 0.0f, gt = 0.0f;
  for (int p = threadIdx.x; p < npatch; p += blockDim.x) {
    const int k = p / nsv, l = p - k * nsv;
    float T[4][4];   // T[a][f] = sum_b P[k+a][l+b] Bv_l[b][f]
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float P = __ldg(ctrl + (k + a) * ncv + (l + b));
        zmn = fminf(zmn, P);
        zmx = fmaxf(zmx, P);
        const float4 q = s.bv[l * 4 + b];
        c0 = fmaf(P, q.x, c0);
        c1 = fmaf(P, q.y, c1);
        c2 = fmaf(P, q.z, c2);
        c3 = fmaf(P, q.w, c3);
      }
      T[a][0] = c0; T[a][1] = c1; T[a][2] = c2; T[a][3] = c3;
    }
    const float4 u0 = s.bu[k * 4 + 0], u1 = s.bu[k * 4 + 1], u2 = s.bu[k * 4 + 2], u3 = s.bu[k * 4 + 3];
    const float ue[4][4] = {{u0.x, u1.x, u2.x, u3.x}, {u0.y, u1.y, u2.y, u3.y},
                            {u0.z, u1.z, u2.z, u3.z}, {u0.w, u1.w, u2.w, u3.w}};  // ue[e][a]
    float4* out = s.patch + (size_t)p * 4;
    float C[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
#pragma unroll
      for (int f = 0; f < 4; ++f)
        C[e][f] = fmaf(ue[e][0], T[0][f], fmaf(ue[e][1], T[1][f], fmaf(ue[e][2], T[2][f], ue[e][3] * T[3][f])));
      out[e] = make_float4(C[e][0], C[e][1], C[e][2], C[e][3]);
    }
    if (s.hull) {
      float ms, mt;
      s.hull[p] = patch_hull(C, &ms, &mt);
      gs = fmaxf(gs, ms);
      gt = fmaxf(gt, mt);
    }
  }
  if (bounds) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zmn = fminf(zmn, __shfl_xor_sync(0xffffffffu, zmn, o));
      zmx = fmaxf(zmx, __shfl_xor_sync(0xffffffffu, zmx, o));
    }
    gs = fmaxf(gs, __shfl_xor_sync(0xffffffffu, gs, 16));
    gs = fmaxf(gs, __shfl_xor_sync(0xffffffffu, gs, 8));
    gs = fmaxf(gs, __shfl_xor_sync(0xffffffffu, gs, 4));
    gs = fmaxf(gs, __shfl_xor_sync(0xffffffffu, gs, 2));
    gs = fmaxf(gs, __shfl_xor_sync(0xffffffffu, gs, 1));
    gt = fmaxf(gt, __shfl_xor_sync(0xffffffffu, gt, 16));
    gt = fmaxf(gt, __shfl_xor_sync(0xffffffffu, gt, 8));
    gt = fmaxf(gt, __shfl_xor_sync(0xffffffffu, gt, 4));
    gt = fmaxf(gt, __shfl_xor_sync(0xffffffffu, gt, 2));
    gt = fmaxf(gt, __shfl_xor_sync(0xffffffffu, gt, 1));
    if ((threadIdx.x & 31) == 0 && zmn <= zmx) {
      atomicMin(&s.zkey[0], float_key(zmn));
      atomicMax(&s.zkey[1], float_key(zmx));
      atomicMax(&s.zkey[2], __float_as_int(gs));   // non-negative floats order as their bits
      atomicMax(&s.zkey[3], __float_as_int(gt));
    }
  }
  __syncthreads();
}

// The exit net's tables (bounds for point sources and two-face lenses).
__device__ inline void build_lens_tables(const Item& it, const LensSmem& s) {
  build_net_tables(it.ctrl, it.ncv, it.nsu, it.nsv, it.kind == FR_SOURCE_POINT || it.two_face, s);
}

// Both nets' tables of a two-face item (the entry net's in `e`).
__device__ inline void build_two_face_tables(const Item& it, const LensSmem& s, const LensSmem& e) {
  build_net_tables(it.ctrl, it.ncv, it.nsu, it.nsv, true, s);
  build_net_tables(it.ctrl_in, it.ncv_in, it.nsu_in, it.nsv_in, true, e);
}

// The exit net's tables of an item at the start of shared memory.
__device__ inline LensSmem carve_exit(unsigned char* base, const Item& it) {
  return carve_lens(base, it.nsu, it.nsv, needs_hull(it));
}

// The entry net's tables follow the exit net's.
__device__ inline LensSmem carve_entry(unsigned char* base, const Item& it) {
  const bool h = needs_hull(it);
  return carve_lens(base + ((lens_smem_bytes(it.nsu, it.nsv, h) + 15) & ~(size_t)15), it.nsu_in, it.nsv_in, h);
}

__device__ __forceinline__ void locate(float u, int ns, int* k, float* s) {
  const float us = fminf(fmaxf(u, 0.0f), 1.0f) * (float)ns;
  const int kk = min((int)us, ns - 1);
  *k = kk;
  *s = us - (float)kk;
}

// One cubic c.x + c.y t + c.z t^2 + c.w t^3 and its derivative.
__device__ __forceinline__ void cubic_d(const float4 c, float t, float* v, float* dv) {
  const float a = fmaf(t, c.w, c.z);
  const float b = fmaf(t, a, c.y);
  const float db = fmaf(t, c.w, a);
  *v = fmaf(t, b, c.x);
  *dv = fmaf(t, db, b);
}

// Z, dZ/ds, dZ/dt of patch q at (s, t).
__device__ __forceinline__ void patch_eval(const float4* q, float s, float t, float* Z, float* Zs, float* Zt) {
  float r0, r1, r2, r3, d0, d1, d2, d3;
  cubic_d(q[0], t, &r0, &d0);
  cubic_d(q[1], t, &r1, &d1);
  cubic_d(q[2], t, &r2, &d2);
  cubic_d(q[3], t, &r3, &d3);
  const float a = fmaf(s, r3, r2);
  const float b = fmaf(s, a, r1);
  const float db = fmaf(s, r3, a);
  *Z = fmaf(s, b, r0);
  *Zs = fmaf(s, db, b);
  *Zt = fmaf(s, fmaf(s, fmaf(s, d3, d2), d1), d0);
}

// d2Z/ds2, d2Z/dsdt, d2Z/dt2 of patch q at (s, t).
__device__ __forceinline__ void patch_eval2(const float4* q, float s, float t, float* Zss, float* Zst, float* Ztt) {
  float r2, r3, d1, d2, d3, tmp;
  cubic_d(q[1], t, &tmp, &d1);
  cubic_d(q[2], t, &r2, &d2);
  cubic_d(q[3], t, &r3, &d3);
  *Zss = fmaf(6.0f * s, r3, 2.0f * r2);
  *Zst = fmaf(s, fmaf(3.0f * s, d3, 2.0f * d2), d1);
  const float4 c0 = q[0], c1 = q[1], c2 = q[2], c3 = q[3];
  const float e0 = fmaf(6.0f * t, c0.w, 2.0f * c0.z);
  const float e1 = fmaf(6.0f * t, c1.w, 2.0f * c1.z);
  const float e2 = fmaf(6.0f * t, c2.w, 2.0f * c2.z);
  const float e3 = fmaf(6.0f * t, c3.w, 2.0f * c3.z);
  *Ztt = fmaf(s, fmaf(s, fmaf(s, e3, e2), e1), e0);
}

// The four non-zero basis functions of a span and their s-derivatives.
__device__ __forceinline__ void basis_eval(const float4* tab, float s, float N[4], float dN[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) cubic_d(tab[a], s, &N[a], &dN[a]);
}

// ---------------------------------------------------------------------------
// One ray up to the screen (Secs. 2.2-2.3); forward and adjoint run this code.
// ---------------------------------------------------------------------------
// Status of a ray whose intersection a hot trace kernel leaves to the deferred
// pass (first_root<false> returned ROOT_DEFER); never reported: that pass
// traces the ray again and counts its real status.
constexpr int kRayDeferred = FR_RAY_NCAUSES - 1;

struct RayFwd {
  int status;
  int iters;
  int k, l;             // patch (knot span product) of the hit
  float u, v;           // hit in the B-spline parameter domain
  float s, t;           // patch coordinates of the hit
  float x, y, z;        // hit on the freeform
  float dx, dy, dz;     // direction inside the glass
  float Zs, Zt;         // surface derivatives in patch coordinates at the hit
  float nx, ny, nz;     // unit normal (into the air)
  float invL;           // 1/|(-Z_x,-Z_y,1)|
  float c, cs, a;       // cos(incidence) d.n, cos(transmission), eta c - cs
  float tx, ty, tz;     // direction after the freeform
  float T1, T2, w;      // Schlick transmissions and final weight
  float lam;            // distance parameter to the screen
  float X, Y;           // screen hit
  float tstar, gp;      // point source: ray parameter of the hit and df/dt there
  int mK, mL, mup;      // triangle mesh: cell and triangle (0 lower-left, 1 upper-right) of the hit
  float ma, mb;         // triangle mesh: the hit in the cell's local coordinates
};

// Exit face: normal, Snell glass -> air, TIR, Schlick, propagation (a5, a6).
// COLL: the ray travels along (0,0,1) inside the glass.
template <bool COLL>
__device__ __forceinline__ void exit_and_propagate(const Item& it, RayFwd& r) {
  const float Zx = r.Zs * it.ku, Zy = r.Zt * it.kv;
  const float q2 = fmaf(Zx, Zx, Zy * Zy);
  const float invL = rsqrtf(1.0f + q2);
  r.invL = invL;
  r.nx = -Zx * invL;
  r.ny = -Zy * invL;
  r.nz = invL;
  const float eta = it.n_glass;
  float c, sin2;
  if (COLL) {
    c = invL;
    sin2 = q2 * invL * invL;            // 1 - c^2 without cancellation
  } else {
    c = fmaf(r.dx, r.nx, fmaf(r.dy, r.ny, r.dz * r.nz));
    sin2 = fmaf(-c, c, 1.0f);
  }
  r.c = c;
  const float k = fmaf(-eta * eta, sin2, 1.0f);
  if (!(k > 0.0f)) { r.status = FR_RAY_TIR; return; }
  const float cs = k * rsqrtf(k);
  r.cs = cs;
  const float a = fmaf(eta, c, -cs);
  r.a = a;
  if (COLL) {
    r.tx = -a * r.nx;
    r.ty = -a * r.ny;
    r.tz = fmaf(-a, r.nz, eta);
  } else {
    r.tx = fmaf(eta, r.dx, -a * r.nx);
    r.ty = fmaf(eta, r.dy, -a * r.ny);
    r.tz = fmaf(eta, r.dz, -a * r.nz);
  }
  const float om = 1.0f - cs;
  const float om2 = om * om;
  r.T2 = (1.0f - it.R0) * fmaf(-om2 * om2, om, 1.0f);
  r.w = it.omega0 * r.T1 * r.T2;
  if (!(r.tz > 0.0f)) { r.status = FR_RAY_OFF_SCREEN; return; }
  const float lam = (it.z_screen - r.z) * fast_rcp(r.tz);
  r.lam = lam;
  r.X = fmaf(lam, r.tx, r.x);
  r.Y = fmaf(lam, r.ty, r.y);
  r.status = (fabsf(r.X) < it.Rx && fabsf(r.Y) < it.Ry) ? FR_RAY_ON_SCREEN : FR_RAY_OFF_SCREEN;
}

// Collimated ray through the freeform at (u, v) = ((x/rx+1)/2, (y/ry+1)/2)
// given Z and its slopes.
__device__ __forceinline__ void collimated_at(const Item& it, float u, float v, float y, float Z, float Zs,
                                              float Zt, RayFwd& r) {
  r.u = u;
  r.v = v;
  r.x = fmaf(2.0f, u, -1.0f) * it.rx;
  r.y = y;
  r.z = Z;
  r.Zs = Zs;
  r.Zt = Zt;
  r.dx = 0.0f;
  r.dy = 0.0f;
  r.dz = 1.0f;
  r.T1 = 1.0f - it.R0;   // normal incidence on the flat entry face
  r.iters = 0;
  exit_and_propagate<true>(it, r);
}

// Collimated ray (a1, a3-a6) on the square grid, any patch (jittered rays).
__device__ __forceinline__ void trace_collimated(const Item& it, const LensSmem& ls, uint32_t row, uint32_t col,
                                                 uint64_t id, float inv_cols, float inv_rows, RayFwd& r) {
  float ja = 0.5f, jb = 0.5f;
  if (it.jitter) {
    const uint2 w = philox_ray_words(it.seed, id);
    ja = unit23(w.x);
    jb = unit23(w.y);
  }
  const float u = ((float)col + ja) * inv_cols;
  const float v = ((float)row + jb) * inv_rows;
  locate(u, it.nsu, &r.k, &r.s);
  locate(v, it.nsv, &r.l, &r.t);
  float Z, Zs, Zt;
  patch_eval(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Z, &Zs, &Zt);
  collimated_at(it, u, v, fmaf(2.0f, v, -1.0f) * it.ry, Z, Zs, Zt, r);
}

// Collimated cell-centre rays along one grid row: t (and with it the v
// basis) is fixed, and u = (col + 1/2)/cols advances by 1/cols from ray to
// ray. The walk takes u in span units, us = u nsu = (col + 1/2) nsu / cols,
// keeps the current patch k (stepped when us passes its right knot, no
// per-ray span search) and the row cubics of that patch,
// r_e(t) = sum_f C[e][f] t^f and their t-derivatives, which serve every ray of
// the row in it.
struct RowWalk {
  int k, l;
  float v, t, y;
  uint32_t col0;        // the first cell's column
  float dus, hdus, kf;  // us step per column, half of it, k as a float
  float r0, r1, r2, r3, d0, d1, d2, d3;

  __device__ __forceinline__ void load(const Item& it, const LensSmem& ls) {
    const float4* q = ls.patch + (size_t)(k * it.nsv + l) * 4;
    cubic_d(q[0], t, &r0, &d0);
    cubic_d(q[1], t, &r1, &d1);
    cubic_d(q[2], t, &r2, &d2);
    cubic_d(q[3], t, &r3, &d3);
  }

  // The walk from cell (row, col).
  __device__ __forceinline__ void begin(const Item& it, const LensSmem& ls, uint32_t row, uint32_t col,
                                        float inv_cols, float inv_rows) {
    v = ((float)row + 0.5f) * inv_rows;
    y = fmaf(2.0f, v, -1.0f) * it.ry;
    locate(v, it.nsv, &l, &t);
    col0 = col;
    dus = inv_cols * (float)it.nsu;
    hdus = 0.5f * dus;
    k = min((int)fmaf((float)col, dus, hdus), it.nsu - 1);
    kf = (float)k;
    load(it, ls);
  }

  // The j-th ray of the walk. us is a function of the ray's column alone (the
  // same rounding whichever lane traces it: deterministic mode stays bit-exact
  // across schedules).
  __device__ __forceinline__ void trace(const Item& it, const LensSmem& ls, uint32_t j, RayFwd& r) {
    const float us = fmaf((float)(col0 + j), dus, hdus);
    if (us >= kf + 1.0f && k < it.nsu - 1) {
      do {
        ++k;
        kf += 1.0f;
      } while (us >= kf + 1.0f && k < it.nsu - 1);
      load(it, ls);
    }
    const float s = us - kf;
    r.k = k;
    r.l = l;
    r.s = s;
    r.t = t;
    const float a = fmaf(s, r3, r2);
    const float b = fmaf(s, a, r1);
    const float db = fmaf(s, r3, a);
    const float Z = fmaf(s, b, r0);
    const float Zs = fmaf(s, db, b);
    const float Zt = fmaf(s, fmaf(s, fmaf(s, d3, d2), d1), d0);
    r.u = us * (1.0f / (float)it.nsu);
    r.v = v;
    r.x = fmaf(us, 2.0f * it.rx / (float)it.nsu, -it.rx);
    r.y = y;
    r.z = Z;
    r.Zs = Zs;
    r.Zt = Zt;
    r.dx = 0.0f;
    r.dy = 0.0f;
    r.dz = 1.0f;
    r.T1 = 1.0f - it.R0;   // normal incidence on the flat entry face
    r.iters = 0;
    exit_and_propagate<true>(it, r);
  }
};

// The adjoint's walk along a lane's run of cells (the forward's is RowWalk in
// column lockstep): along one grid row t is fixed: the row cubics of the current patch,
// r_e(t) = sum_f C[e][f] t^f and their t-derivatives, serve every ray of the
// row that falls in that patch.
struct RowPatch {
  uint32_t row;
  int k, l;
  float v, t, y;
  float r0, r1, r2, r3, d0, d1, d2, d3;
};

__device__ __forceinline__ void row_patch_load(const Item& it, const LensSmem& ls, int k, RowPatch& rp) {
  const float4* q = ls.patch + (size_t)(k * it.nsv + rp.l) * 4;
  cubic_d(q[0], rp.t, &rp.r0, &rp.d0);
  cubic_d(q[1], rp.t, &rp.r1, &rp.d1);
  cubic_d(q[2], rp.t, &rp.r2, &rp.d2);
  cubic_d(q[3], rp.t, &rp.r3, &rp.d3);
  rp.k = k;
}

// Collimated ray at a cell centre, with the row cache.
__device__ __forceinline__ void trace_collimated_row(const Item& it, const LensSmem& ls, uint32_t row, uint32_t col,
                                                     float inv_cols, float inv_rows, RowPatch& rp, RayFwd& r) {
  if (row != rp.row) {
    rp.row = row;
    rp.v = ((float)row + 0.5f) * inv_rows;
    rp.y = fmaf(2.0f, rp.v, -1.0f) * it.ry;
    locate(rp.v, it.nsv, &rp.l, &rp.t);
    rp.k = -1;
  }
  const float u = ((float)col + 0.5f) * inv_cols;
  int k;
  locate(u, it.nsu, &k, &r.s);
  if (k != rp.k) row_patch_load(it, ls, k, rp);
  r.k = k;
  r.l = rp.l;
  r.t = rp.t;
  const float s = r.s;
  const float a = fmaf(s, rp.r3, rp.r2);
  const float b = fmaf(s, a, rp.r1);
  const float db = fmaf(s, rp.r3, a);
  const float Z = fmaf(s, b, rp.r0);
  const float Zs = fmaf(s, db, b);
  const float Zt = fmaf(s, fmaf(s, fmaf(s, rp.d3, rp.d2), rp.d1), rp.d0);
  collimated_at(it, u, rp.v, rp.y, Z, Zs, Zt, r);
}

// Collimated cell-centre rays in column lockstep (forward trace): the rows of the call's cell range are taken in blocks of 32, one
// row per lane, and the columns of the blocks, block after block, are split
// evenly over the item's warps. At every step the lanes of a warp trace the
// same column of 32 neighbouring rows, so their footprints move on to the next
// pixel column, and their rays into the next patch, at nearly the same step:
// the register sums are flushed, the dL/dE footprint re-read and the patch
// cubics loaded by the whole warp at once rather than lane after lane.
struct Lockstep {
  uint64_t s, s1;   // this warp's column steps [s, s1)

  // The column steps of the call's rows: blocks of 32 rows times the columns.
  static __device__ __forceinline__ uint64_t steps(const Item& it) {
    return (uint64_t)((it.row_hi - it.row_lo + 31) / 32) * (uint64_t)it.cols;
  }

  __device__ __forceinline__ void init(const Item& it, int warps) {
    const uint64_t S = steps(it);
    const uint64_t W = (uint64_t)(it.cta_end - it.cta_begin) * (uint64_t)warps;
    const uint64_t gw = (uint64_t)((int)blockIdx.x - it.cta_begin) * (uint64_t)warps + (threadIdx.x >> 5);
    s = S * gw / W;
    s1 = S * (gw + 1) / W;
  }

  // The next run of this lane, cells (row, col + j) for j in [j0, j1) (empty
  // for a lane past the last row or outside the call's range); false when the
  // warp's share is done. Every lane of a warp returns the same col.
  __device__ __forceinline__ bool next(const Item& it, uint32_t* row, uint32_t* col, uint32_t* j0, uint32_t* j1) {
    if (s >= s1) return false;
    const uint32_t cols = (uint32_t)it.cols;
    const uint32_t rb = (uint32_t)(s / cols);
    const uint32_t c0 = (uint32_t)(s - (uint64_t)rb * cols);
    const uint32_t n = (uint32_t)min((uint64_t)(cols - c0), s1 - s);
    s += n;
    const uint32_t r = it.row_lo + rb * 32u + (threadIdx.x & 31u);
    uint32_t a = 0, b = r < it.row_hi ? n : 0u;
    if (r == it.row_lo && it.col_lo > c0) a = min(it.col_lo - c0, n);
    if (r + 1 == it.row_hi) b = it.col_hi > c0 ? min(it.col_hi - c0, b) : 0u;
    *row = r;
    *col = c0;
    *j0 = a;
    *j1 = max(a, b);
    return true;
  }

  // Most cells one CTA of `warps` warps can take (for fixed-point bounds).
  static __device__ __forceinline__ uint64_t max_per_cta(const Item& it, int warps) {
    const uint64_t S = steps(it);
    const uint64_t W = (uint64_t)(it.cta_end - it.cta_begin) * (uint64_t)warps;
    const uint64_t ci = (uint64_t)((int)blockIdx.x - it.cta_begin);
    return 32 * (S * (ci + 1) * warps / W - S * ci * warps / W);
  }
};

// f(t) = Z(o_uv + d_uv t) - o_z - d_z t (Eq. surfaceintersect) and df/dt.
__device__ __forceinline__ void f_eval(const Item& it, const LensSmem& ls, float ou, float ov, float du, float dv,
                                       float oz, float dz, float t, RayFwd& r, float* f, float* fp) {
  locate(fmaf(du, t, ou), it.nsu, &r.k, &r.s);
  locate(fmaf(dv, t, ov), it.nsv, &r.l, &r.t);
  float Z;
  patch_eval(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Z, &r.Zs, &r.Zt);
  *f = Z - fmaf(dz, t, oz);
  *fp = fmaf(r.Zs, du * (float)it.nsu, fmaf(r.Zt, dv * (float)it.nsv, -dz));
}

// ---------------------------------------------------------------------------
// Sec. 2.2.1, Eq. surfaceintersect: the hit is the SMALLEST positive root of
// f(t) = Z(o_uv + d_uv t) - o_z - d_z t over the domain. f > 0 while the ray is
// below the surface. The root is found in two phases:
//  1. A certified march from the bottom of the convex-hull slab: the patches
//     (knot span products) the ray's (u, v) path crosses are visited in order
//     of t; a patch whose lowest point (patch_hull) the ray only reaches after
//     leaving it holds no root and is skipped; inside a patch, from a point t
//     with f(t) > 0 and slope g = f'(t), the bound |f''| <= M of patch_hull
//     gives f(t + d) >= f(t) + g d - M d^2 / 2 > 0 for every d below the
//     positive root d* of that quadratic, so [t, t + d*) holds no root and the
//     march moves to t + d*. (For a transverse root d* tends to the Newton step:
//     the march converges quadratically from the left.)
//  2. As soon as g < 0 and 2 M f < g^2, f is strictly decreasing on
//     [t, t + 2f/|g|] (f' <= g + 2 M f/|g| < 0 there) and negative at its end,
//     so that interval holds exactly one root, the first: safeguarded Newton
//     (at most newton_max iterations, until a step is below the tolerance) runs
//     on that bracket. When the bracket would reach past the patch, f at the
//     patch's edge decides whether the root lies before it.
// ---------------------------------------------------------------------------

// The ray's (u, v, z) as functions of its parameter t on one net.
struct NetLine {
  float ou, ov, du, dv, oz, dz;
};

enum { ROOT_FOUND = 0, ROOT_NONE = 1, ROOT_FAIL = 2, ROOT_DEFER = 3 };

// Evaluations the march may take before Newton's bracket is found.
constexpr int kMarchMax = 32;   // evaluations of the march, besides Newton's

// The walk over the patches of one net along the ray: the current patch
// (k, l), where the ray leaves it (tx, and whether through a u edge), and the
// bound M of |f''| on it (patch_hull).
struct PatchWalk {
  int k, l;
  float tx, M;
  bool exit_u;

  // Enters patch (k, l) at t: sets tx and M, and returns the first t in the
  // patch that may be a root (the ray reaching the patch's lowest point).
  __device__ __forceinline__ float enter(const float4* hull, int nsv, const NetLine& q, float inv_du, float inv_dv,
                                         float inv_ns_u, float inv_ns_v, float inv_dz, float a2, float b2, float t,
                                         float tb) {
    const float txu = q.du != 0.0f ? ((float)(k + (q.du > 0.0f ? 1 : 0)) * inv_ns_u - q.ou) * inv_du : INFINITY;
    const float txv = q.dv != 0.0f ? ((float)(l + (q.dv > 0.0f ? 1 : 0)) * inv_ns_v - q.ov) * inv_dv : INFINITY;
    exit_u = txu <= txv;
    tx = fminf(fminf(txu, txv), tb);
    const float4 h = hull[k * nsv + l];
    M = fmaf(h.z, a2, h.w * b2);
    return fmaxf(t, (h.x - q.oz) * inv_dz);
  }
};

// f(t) and f'(t) on a net whose power-form patches are `patch` (the same
// arithmetic as f_eval and f_eval_in, without a ray record).
__device__ __forceinline__ void net_f(const float4* patch, int nsu, int nsv, const NetLine& q, float t, float* f,
                                      float* fp) {
  int k, l;
  float s, u, Z, Zs, Zt;
  locate(fmaf(q.du, t, q.ou), nsu, &k, &s);
  locate(fmaf(q.dv, t, q.ov), nsv, &l, &u);
  patch_eval(patch + (size_t)(k * nsv + l) * 4, s, u, &Z, &Zs, &Zt);
  *f = Z - fmaf(q.dz, t, q.oz);
  *fp = fmaf(Zs, q.du * (float)nsu, fmaf(Zt, q.dv * (float)nsv, -q.dz));
}

// The march: the smallest root of f on [ta, tb] (f(ta) >= 0): ROOT_FOUND
// with t, ROOT_NONE when the ray reaches tb first, ROOT_FAIL when the march or
// Newton runs out of evaluations. One loop with one evaluation per pass
// serves both phases, so that the lanes of a warp evaluate together whichever
// phase each is in. Out of line: the quick path (first_root) rarely needs it.
static __device__ __noinline__ int first_root_march(const float4* patch, const float4* hull, int nsu, int nsv, NetLine q,
                                             float ta, float tb, int newton_max, float tol, float* t_out, int* iters) {
  const float fnsu = (float)nsu, fnsv = (float)nsv;
  const float a = q.du * fnsu, b = q.dv * fnsv;   // ds/dt, dt/dt in patch units
  const float a2 = a * a, b2 = b * b;
  const float inv_dz = fast_rcp(q.dz);
  const float inv_du = q.du != 0.0f ? fast_rcp(q.du) : 0.0f, inv_dv = q.dv != 0.0f ? fast_rcp(q.dv) : 0.0f;
  const float inv_ns_u = fast_rcp(fnsu), inv_ns_v = fast_rcp(fnsv);
  PatchWalk w;
  w.k = min(max((int)(fmaf(q.du, ta, q.ou) * fnsu), 0), nsu - 1);
  w.l = min(max((int)(fmaf(q.dv, ta, q.ov) * fnsv), 0), nsv - 1);
  *iters = 0;
  // The first patch that may hold a root; a patch whose lowest point the ray
  // only reaches after leaving it is passed without an evaluation.
  float t = w.enter(hull, nsv, q, inv_du, inv_dv, inv_ns_u, inv_ns_v, inv_dz, a2, b2, ta, tb);
  for (int visit = 0; t >= w.tx; ++visit) {
    if (w.tx >= tb || visit > nsu + nsv) return ROOT_NONE;
    if (w.exit_u) w.k += q.du > 0.0f ? 1 : -1;
    else w.l += q.dv > 0.0f ? 1 : -1;
    if (w.k < 0 || w.k >= nsu || w.l < 0 || w.l >= nsv) return ROOT_NONE;
    t = w.enter(hull, nsv, q, inv_du, inv_dv, inv_ns_u, inv_ns_v, inv_dz, a2, b2, w.tx, tb);
  }
  int phase = 0;   // 0 march, 1 f at the patch's edge, 2 Newton on [lo, hi]
  float lo = t, hi = t, flo = 0.0f, glo = 0.0f, tprev = t;
  int nn = 0;
  for (int pass = 0; pass < kMarchMax + newton_max; ++pass) {
    float f, g;
    net_f(patch, nsu, nsv, q, t, &f, &g);
    if (phase == 2) {
      ++nn;
      if (f > 0.0f) lo = t; else hi = t;
      if (fabsf(t - tprev) <= tol || f == 0.0f) {
        *t_out = t;
        *iters = nn;
        return ROOT_FOUND;
      }
      if (nn >= newton_max) return ROOT_FAIL;
      float tn = t - __fdividef(f, g);
      // The bracket is closed: an exact root on its edge (Newton landing on the
      // root leaves f within rounding of 0 on either side) is kept, not bisected.
      if (!(g < 0.0f) || !(tn >= lo && tn <= hi)) tn = 0.5f * (lo + hi);
      tprev = t;
      t = tn;
      continue;
    }
    if (phase == 1) {   // f at the edge of a patch on which f decreases strictly from lo
      if (f == 0.0f) {
        *t_out = t;
        return ROOT_FOUND;
      }
      if (f < 0.0f) {   // the root lies in [lo, edge]: Newton from lo
        phase = 2;
        hi = t;
        float tn = lo - __fdividef(flo, glo);
        if (!(tn >= lo && tn <= hi)) tn = 0.5f * (lo + hi);
        tprev = lo;
        t = tn;
        continue;
      }
      phase = 0;   // no root up to the edge: on to the next patch
    } else {
      if (!(f > 0.0f)) {   // on the root within rounding
        *t_out = t;
        return ROOT_FOUND;
      }
      if (g < 0.0f && 2.0f * w.M * f < g * g) {
        // f decreases strictly on [t, t + 2f/|g|] and is negative at its end
        const float n = f * fast_rcp(-g);
        lo = t;
        if (t + 2.0f * n <= w.tx) {
          phase = 2;
          hi = t + 2.0f * n;
          tprev = t;
          t += n;   // the first Newton step
        } else {
          phase = 1;
          flo = f;
          glo = g;
          t = w.tx;
        }
        continue;
      }
      // certified step: f + g d - M d^2 / 2 > 0 for 0 <= d < d*
      const float r = fast_sqrt(fmaf(g, g, 2.0f * w.M * f));
      t += g <= 0.0f ? 2.0f * f * fast_rcp(r - g) : (w.M > 0.0f ? (g + r) * fast_rcp(w.M) : INFINITY);
      if (t < w.tx) continue;
    }
    // leave the patch at its edge; pass the patches the ray stays below
    t = w.tx;
    for (int visit = 0; t >= w.tx; ++visit) {
      if (w.tx >= tb || visit > nsu + nsv) return ROOT_NONE;
      if (w.exit_u) w.k += q.du > 0.0f ? 1 : -1;
      else w.l += q.dv > 0.0f ? 1 : -1;
      if (w.k < 0 || w.k >= nsu || w.l < 0 || w.l >= nsv) return ROOT_NONE;
      t = w.enter(hull, nsv, q, inv_du, inv_dv, inv_ns_u, inv_ns_v, inv_dz, a2, b2, w.tx, tb);
    }
  }
  return ROOT_FAIL;
}

// Whether [ta, te) holds no root of f, given f(te) = fe >= 0 and f'(te) = ge
// (te a root Newton found, fe = 0, or the side of the domain, fe > 0), from the
// patch bounds alone (no evaluation of f): the patches the ray crosses before
// the first one whose lowest point it reaches (tc) hold none, and from tc on,
// with |f''| <= Mmax over every patch crossed, f(t) >= q(d) = fe - ge d -
// Mmax d^2 / 2 for d = te - t; q is concave, so q > 0 on [0, te - tc] follows
// from q(0) = fe >= 0 (and ge < 0 when fe = 0) and q(te - tc) > 0.
__device__ __forceinline__ bool no_root_before(const float4* hull, int nsu, int nsv, const NetLine& q, float ta,
                                               float te, float fe, float ge) {
  if (!(fe > 0.0f) && !(fe == 0.0f && ge < 0.0f)) return false;
  // a margin of 12% on the curvature bound for the rounding of f, f' and the bounds in FP32
  auto holds = [&](float D, float M) { return fe - ge * D - 0.56f * M * D * D > 0.0f; };
  const float fnsu = (float)nsu, fnsv = (float)nsv;
  const float a = q.du * fnsu, b = q.dv * fnsv;
  const float a2 = a * a, b2 = b * b;
  const float inv_dz = fast_rcp(q.dz);
  {   // the usual case: the ray is over one patch from ta to te
    const int k0 = min(max((int)(fmaf(q.du, ta, q.ou) * fnsu), 0), nsu - 1);
    const int l0 = min(max((int)(fmaf(q.dv, ta, q.ov) * fnsv), 0), nsv - 1);
    const int k1 = min(max((int)(fmaf(q.du, te, q.ou) * fnsu), 0), nsu - 1);
    const int l1 = min(max((int)(fmaf(q.dv, te, q.ov) * fnsv), 0), nsv - 1);
    if (k0 == k1 && l0 == l1) {
      const float4 h = hull[k1 * nsv + l1];
      const float tc = fmaxf(ta, (h.x - q.oz) * inv_dz);
      return tc >= te || holds(te - tc, fmaf(h.z, a2, h.w * b2));
    }
  }
  const float inv_du = q.du != 0.0f ? fast_rcp(q.du) : 0.0f, inv_dv = q.dv != 0.0f ? fast_rcp(q.dv) : 0.0f;
  PatchWalk w;
  w.k = min(max((int)(fmaf(q.du, ta, q.ou) * fnsu), 0), nsu - 1);
  w.l = min(max((int)(fmaf(q.dv, ta, q.ov) * fnsv), 0), nsv - 1);
  float t = ta, tc = INFINITY, Mmax = 0.0f;
  for (int visit = 0; visit <= nsu + nsv; ++visit) {
    const float tz = w.enter(hull, nsv, q, inv_du, inv_dv, 1.0f / fnsu, 1.0f / fnsv, inv_dz, a2, b2, t, te);
    if (tc < INFINITY || tz < w.tx) {   // from the first patch the ray may meet on
      tc = fminf(tc, tz);
      Mmax = fmaxf(Mmax, w.M);
    }
    if (w.tx >= te) break;
    t = w.tx;
    if (w.exit_u) w.k += q.du > 0.0f ? 1 : -1;
    else w.l += q.dv > 0.0f ? 1 : -1;
    if (w.k < 0 || w.k >= nsu || w.l < 0 || w.l >= nsv) break;
  }
  return tc >= te || holds(te - tc, Mmax);
}

// The smallest root of f on [ta, tb] (f(ta) >= 0), as first_root_march
// defines it, found the quick way where that is safe. When the net's slope
// bounds (gs >= |Z_s|, gt >= |Z_t|) make f strictly decreasing along the
// whole ray (gs |ds/dt| + gt |dt/dt| < d_z), f has at most one root: f(tb) > 0
// at a side of the domain means none, else safeguarded Newton from the middle
// of [ta, tb] finds it. Otherwise the patch bounds must certify the result
// (no_root_before): that no root lies before the one Newton found, or before
// the side. Where that fails, or Newton does not converge, the march decides
// (MARCH), or the ray is handed back as ROOT_DEFER for a later pass that
// marches (the hot kernels keep the march's code out of their loops).
template <bool MARCH, class Eval>
__device__ __forceinline__ int first_root(const float4* patch, const float4* hull, int nsu, int nsv, const NetLine& q,
                                          float ta, float tb, bool tb_is_top, float gs, float gt, int newton_max,
                                          float tol, Eval eval, float* t_out, float* fp_out, int* iters) {
  const bool mono = fmaf(gs, fabsf(q.du * (float)nsu), gt * fabsf(q.dv * (float)nsv)) < 0.999f * q.dz;
  float f, g;
  bool bracketed = true;
  if (!tb_is_top) {   // the slab's top has f <= 0 (convex hull); a side of the domain may not
    eval(tb, &f, &g);
    bracketed = !(f > 0.0f);
    // the ray leaves through the side with f > 0: no root if f is monotone, or
    // if the bounds show none before
    if (!bracketed && (mono || no_root_before(hull, nsu, nsv, q, ta, tb, f, g))) return ROOT_NONE;
  }
  if (bracketed) {
    float lo = ta, hi = tb;
    float t = 0.5f * (ta + tb);
    eval(t, &f, &g);
    if (f > 0.0f) lo = t; else hi = t;
    bool converged = (f == 0.0f);
    int n = 0;
    for (; n < newton_max && !converged; ++n) {
      float tn = t - __fdividef(f, g);
      // The bracket is closed: an exact root on its edge (Newton landing on the
      // root leaves f within rounding of 0 on either side) is kept, not bisected.
      if (!(g < 0.0f) || !(tn >= lo && tn <= hi)) tn = 0.5f * (lo + hi);
      const float step = fabsf(tn - t);
      t = tn;
      eval(t, &f, &g);
      if (f > 0.0f) lo = t; else hi = t;
      if (step <= tol || f == 0.0f) converged = true;
    }
    if (converged && (mono || no_root_before(hull, nsu, nsv, q, ta, t, 0.0f, g))) {
      *t_out = t;
      *fp_out = g;
      *iters = n;
      return ROOT_FOUND;
    }
  }
  if constexpr (!MARCH) {
    return ROOT_DEFER;
  } else {
    const int st = first_root_march(patch, hull, nsu, nsv, q, ta, tb, newton_max, tol, t_out, iters);
    if (st == ROOT_FOUND) eval(*t_out, &f, fp_out);   // the caller's record at the root
    return st;
  }
}

// ---------------------------------------------------------------------------
// Sec. 2.2.2: the triangle mesh. Knot span product (k, l) is split into
// mesh_nu x mesh_nv rectangles; with uniform knots all rectangles form one grid
// of NU x NV cells over [0,1]^2. With local coordinates a = NU u - K,
// b = NV v - L, cell (K, L) has a lower-left triangle {a >= 0, b >= 0,
// a + b < 1} and an upper-right one {a < 1, b < 1, a + b >= 1}; on each the
// mesh is the plane through its three vertices, which lie on the surface
// (Eq. trianglefuncdetermined).
// ---------------------------------------------------------------------------

// Heights of the four corners of cell (K, L) from the power form of its patch.
__device__ __forceinline__ void cell_nodes(const Item& it, const LensSmem& ls, int K, int L, float* z00, float* z10,
                                           float* z01, float* z11) {
  const int k = K / it.mesh_nu, l = L / it.mesh_nv;
  const float s0 = (float)(K - k * it.mesh_nu) * it.inv_mnu, s1 = s0 + it.inv_mnu;
  const float t0 = (float)(L - l * it.mesh_nv) * it.inv_mnv, t1 = t0 + it.inv_mnv;
  const float4* q = ls.patch + (size_t)(k * it.nsv + l) * 4;
  float r0[4], r1[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float4 c = q[e];
    r0[e] = fmaf(t0, fmaf(t0, fmaf(t0, c.w, c.z), c.y), c.x);
    r1[e] = fmaf(t1, fmaf(t1, fmaf(t1, c.w, c.z), c.y), c.x);
  }
  *z00 = fmaf(s0, fmaf(s0, fmaf(s0, r0[3], r0[2]), r0[1]), r0[0]);
  *z10 = fmaf(s1, fmaf(s1, fmaf(s1, r0[3], r0[2]), r0[1]), r0[0]);
  *z01 = fmaf(s0, fmaf(s0, fmaf(s0, r1[3], r1[2]), r1[1]), r1[0]);
  *z11 = fmaf(s1, fmaf(s1, fmaf(s1, r1[3], r1[2]), r1[1]), r1[0]);
}

// The plane of a triangle as z = c0 + ca a + cb b.
__device__ __forceinline__ void tri_plane(float z00, float z10, float z01, float z11, int upper, float* c0, float* ca,
                                          float* cb) {
  if (!upper) {
    *ca = z10 - z00;
    *cb = z01 - z00;
    *c0 = z00;
  } else {   // z11 + (z11 - z01)(a - 1) + (z11 - z10)(b - 1)
    *ca = z11 - z01;
    *cb = z11 - z10;
    *c0 = z11 - *ca - *cb;
  }
}

// Mesh height at (u, v) in [0,1]^2.
__device__ __forceinline__ float mesh_height(const Item& it, const LensSmem& ls, float u, float v) {
  const int K = min(max((int)floorf(u * (float)it.NU), 0), it.NU - 1);
  const int L = min(max((int)floorf(v * (float)it.NV), 0), it.NV - 1);
  const float a = fmaf(u, (float)it.NU, -(float)K), b = fmaf(v, (float)it.NV, -(float)L);
  float z00, z10, z01, z11, c0, ca, cb;
  cell_nodes(it, ls, K, L, &z00, &z10, &z01, &z11);
  tri_plane(z00, z10, z01, z11, a + b >= 1.0f ? 1 : 0, &c0, &ca, &cb);
  return fmaf(ca, a, fmaf(cb, b, c0));
}

// First triangle along the ray (u, v, z)(t) = (ou + du t, ov + dv t, oz + dz t)
// for t in [ta, tb]: the cells its (u,v) path crosses are visited in order of
// t (a grid walk), each cell's two triangles tested; the first cell with a hit
// holds the first hit. The inside test has a margin of 1e-4 cell widths so that
// FP32 rounding cannot let a ray slip between two triangles; near an edge both
// may accept and the smaller t is kept; no hit is taken past tb (the side of
// the lens or the top of the slab). At most NU + NV cells are visited. On
// a hit fills tstar, gp (= dg/dt of g = mesh - ray height), the cell,
// triangle and local coordinates, and the cell count in iters.
__device__ __forceinline__ bool mesh_intersect(const Item& it, const LensSmem& ls, float ou, float ov, float du,
                                               float dv, float oz, float dz, float ta, float tb, RayFwd& r) {
  const float fNU = (float)it.NU, fNV = (float)it.NV;
  int K = min(max((int)floorf(fmaf(du, ta, ou) * fNU), 0), it.NU - 1);
  int L = min(max((int)floorf(fmaf(dv, ta, ov) * fNV), 0), it.NV - 1);
  const float da = du * fNU, db = dv * fNV;      // d(a)/dt, d(b)/dt
  const int sK = du > 0.0f ? 1 : -1, sL = dv > 0.0f ? 1 : -1;
  float tK = INFINITY, tL = INFINITY, dtK = INFINITY, dtL = INFINITY;
  if (du != 0.0f) {
    tK = ((float)(K + (du > 0.0f ? 1 : 0)) / fNU - ou) / du;
    dtK = 1.0f / fabsf(da);
  }
  if (dv != 0.0f) {
    tL = ((float)(L + (dv > 0.0f ? 1 : 0)) / fNV - ov) / dv;
    dtL = 1.0f / fabsf(db);
  }
  constexpr float eps = 1e-4f;
  const int max_cells = it.NU + it.NV;
  for (int n = 0; n < max_cells; ++n) {
    float z00, z10, z01, z11;
    cell_nodes(it, ls, K, L, &z00, &z10, &z01, &z11);
    const float a0 = fmaf(fNU, ou, -(float)K), b0 = fmaf(fNV, ov, -(float)L);
    float best = INFINITY;
#pragma unroll
    for (int up = 0; up < 2; ++up) {
      float c0, ca, cb;
      tri_plane(z00, z10, z01, z11, up, &c0, &ca, &cb);
      // c0 + ca (a0 + da t) + cb (b0 + db t) = oz + dz t
      const float den = dz - fmaf(ca, da, cb * db);
      const float t = (fmaf(ca, a0, fmaf(cb, b0, c0)) - oz) / den;
      // The hit must lie over the domain: the inside test's margin must not
      // accept a point past the side of the lens (t > tb) on a boundary cell.
      if (!(t >= 0.0f) || !(t < best) || !(t <= tb)) continue;
      const float a = fmaf(da, t, a0), b = fmaf(db, t, b0);
      const bool in = up ? (a <= 1.0f + eps && b <= 1.0f + eps && a + b >= 1.0f - eps)
                         : (a >= -eps && b >= -eps && a + b <= 1.0f + eps);
      if (!in) continue;
      best = t;
      r.tstar = t;
      r.gp = -den;
      r.mK = K;
      r.mL = L;
      r.mup = up;
      r.ma = a;
      r.mb = b;
    }
    if (best < INFINITY) {
      r.iters = n + 1;
      return true;
    }
    if (tK < tL) {
      if (tK > tb) break;
      K += sK;
      tK += dtK;
      if (K < 0 || K >= it.NU) break;
    } else {
      if (!(tL <= tb)) break;
      L += sL;
      tL += dtL;
      if (L < 0 || L >= it.NV) break;
    }
  }
  r.iters = max_cells;
  return false;
}

// Weights of the hit height in the control heights: on the mesh the hit lies on
// the triangle's plane, z = sum_v lambda_v Z(u_v, v_v), so
// dz/dP_{kt+a,lt+b} = sum_v lambda_v N_a(u_v) N_b(v_v) over the triangle's three
// vertices (barycentric lambda_v) in the triangle's patch (kt, lt); W[a][b]
// returns that sum. (Within the inside test's margin the triangle's patch can
// be the neighbour of the hit's own.)
__device__ __forceinline__ void mesh_vertex_weights(const Item& it, const LensSmem& ls, const RayFwd& r,
                                                    float (&W)[4][4], int* kt, int* lt) {
  const int k = r.mK / it.mesh_nu, l = r.mL / it.mesh_nv;
  *kt = k;
  *lt = l;
  const float s0 = (float)(r.mK - k * it.mesh_nu) * it.inv_mnu, s1 = s0 + it.inv_mnu;
  const float t0 = (float)(r.mL - l * it.mesh_nv) * it.inv_mnv, t1 = t0 + it.inv_mnv;
  float Nu0[4], Nu1[4], Nv0[4], Nv1[4], tmp[4];
  basis_eval(ls.bu + k * 4, s0, Nu0, tmp);
  basis_eval(ls.bu + k * 4, s1, Nu1, tmp);
  basis_eval(ls.bv + l * 4, t0, Nv0, tmp);
  basis_eval(ls.bv + l * 4, t1, Nv1, tmp);
  // lower-left: (1-a-b) z00 + a z10 + b z01; upper-right: (a+b-1) z11 + (1-a) z01 + (1-b) z10
  const float a = r.ma, b = r.mb;
  float l00 = 0.0f, l10, l01, l11 = 0.0f;
  if (!r.mup) {
    l00 = 1.0f - a - b;
    l10 = a;
    l01 = b;
  } else {
    l11 = a + b - 1.0f;
    l01 = 1.0f - a;
    l10 = 1.0f - b;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float p0 = l00 * Nu0[i], p1 = l10 * Nu1[i];
    const float q0 = l01 * Nu0[i], q1 = l11 * Nu1[i];
#pragma unroll
    for (int j = 0; j < 4; ++j) W[i][j] = fmaf(p0 + p1, Nv0[j], (q0 + q1) * Nv1[j]);
  }
}

// Point source ray (a1): origin (sx, sy, pz) of the emitting source of the
// grid and a direction uniform in the cone; omc = 1 - cos(phi), sphi = sin(phi).
__device__ __forceinline__ void source_ray(const Item& it, uint64_t id, float* sx, float* sy, float* d0x, float* d0y,
                                           float* d0z, float* omc, float* sphi) {
  const uint2 w = philox_ray_words(it.seed, id);
  const float xi1 = unit23(w.x), xi2 = unit23(w.y);
  float x = it.px, y = it.py;
  if (it.gnx * it.gny > 1) {
    uint32_t src = (uint32_t)(id / it.per_src);
    src = min(src, (uint32_t)(it.gnx * it.gny - 1));
    const uint32_t gx = src % (uint32_t)it.gnx, gy = src / (uint32_t)it.gnx;
    x += fmaf((float)gx, it.gdx, it.gx0);
    y += fmaf((float)gy, it.gdy, it.gy0);
  }
  *sx = x;
  *sy = y;
  float sn, cn;
  sincospif(2.0f * xi1, &sn, &cn);
  const float o = it.omc_max * xi2;            // 1 - cos(phi)
  const float sp = sqrtf(o * (2.0f - o));
  *d0x = cn * sp;
  *d0y = sn * sp;
  *d0z = 1.0f - o;
  *omc = o;
  *sphi = sp;
}

// The ray inside the glass, from (ox, oy, oz) along (r.dx, r.dy, r.dz), meets
// the exit freeform (a4): safeguarded Newton on f(t) bracketed by the convex
// hull of the control heights (Sec. 2.1.2), or the triangle mesh; then a5-a6.
template <bool MARCH>
__device__ __forceinline__ void exit_hit(const Item& it, const LensSmem& ls, float ox, float oy, float oz, float zmin,
                                         float zmax, RayFwd& r) {
  // Bracket: the slab zmin <= z <= zmax, widened a little for FP32 rounding,
  // cut where the ray leaves the domain [0,1]^2 (the side of the lens).
  const float pad = 1e-6f * (1.0f + fmaxf(fabsf(zmin), fabsf(zmax)));
  const float inv_dz = fast_rcp(r.dz);
  float ta = fmaxf(0.0f, (zmin - pad - oz) * inv_dz);
  const float t_hi = (zmax + pad - oz) * inv_dz;
  const float ou = fmaf(0.5f / it.rx, ox, 0.5f), ov = fmaf(0.5f / it.ry, oy, 0.5f);
  const float du = r.dx * (0.5f / it.rx), dv = r.dy * (0.5f / it.ry);
  float t_dom = INFINITY;
  if (du > 0.0f) t_dom = fminf(t_dom, (1.0f - ou) / du);
  if (du < 0.0f) t_dom = fminf(t_dom, -ou / du);
  if (dv > 0.0f) t_dom = fminf(t_dom, (1.0f - ov) / dv);
  if (dv < 0.0f) t_dom = fminf(t_dom, -ov / dv);
  if (t_dom < ta) { r.status = FR_RAY_OUT_OF_DOMAIN; return; }
  float tb = fminf(t_hi, t_dom);
  float f, fp;
  if (it.mesh_nu > 0) {
    // Triangle mesh (Sec. 2.2.2) instead of Newton; the normal is still the
    // B-spline's at the hit.
    if (ta == 0.0f && mesh_height(it, ls, fminf(fmaxf(ou, 0.0f), 1.0f), fminf(fmaxf(ov, 0.0f), 1.0f)) < oz) {
      r.status = FR_RAY_INVALID;
      return;
    }
    if (!mesh_intersect(it, ls, ou, ov, du, dv, oz, r.dz, ta, tb, r)) {
      r.status = FR_RAY_OUT_OF_DOMAIN;
      return;
    }
    const float t = r.tstar;
    r.u = fmaf(du, t, ou);
    r.v = fmaf(dv, t, ov);
    r.x = fmaf(r.dx, t, ox);
    r.y = fmaf(r.dy, t, oy);
    r.z = fmaf(r.dz, t, oz);
    locate(r.u, it.nsu, &r.k, &r.s);   // the normal is the B-spline's at the hit itself
    locate(r.v, it.nsv, &r.l, &r.t);
    float Z;
    patch_eval(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Z, &r.Zs, &r.Zt);
    exit_and_propagate<false>(it, r);
    return;
  }
  // f(ta) >= 0 by the convex hull unless the slab starts at the entry face,
  // where the freeform may lie below it.
  if (ta == 0.0f) {
    f_eval(it, ls, ou, ov, du, dv, oz, r.dz, 0.0f, r, &f, &fp);
    if (f < 0.0f) { r.status = FR_RAY_INVALID; return; }
  }
  // The smallest root: certified march, then Newton on a bracket that isolates it.
  const NetLine q{ou, ov, du, dv, oz, r.dz};
  auto eval = [&](float t, float* fv, float* gv) { f_eval(it, ls, ou, ov, du, dv, oz, r.dz, t, r, fv, gv); };
  float t;
  float gs, gt;
  slopes(ls, &gs, &gt);
  const int found = first_root<MARCH>(ls.patch, ls.hull, it.nsu, it.nsv, q, ta, tb, !(tb < t_hi), gs, gt,
                                      it.newton_max, it.newton_tol, eval, &t, &fp, &r.iters);
  if (found == ROOT_NONE) { r.status = FR_RAY_OUT_OF_DOMAIN; return; }   // leaves the side first
  if (found == ROOT_FAIL) { r.status = FR_RAY_NEWTON_FAIL; return; }
  if (found == ROOT_DEFER) { r.status = kRayDeferred; return; }
  r.tstar = t;
  r.gp = fp;
  r.u = fmaf(du, t, ou);
  r.v = fmaf(dv, t, ov);
  r.x = fmaf(r.dx, t, ox);
  r.y = fmaf(r.dy, t, oy);
  r.z = fmaf(r.dz, t, oz);
  exit_and_propagate<false>(it, r);
}

// Point source (a1, a2, a4-a6): Philox direction uniform in the cone, flat
// entry face, Snell + Schlick into the glass, then the exit freeform.
template <bool MARCH>
__device__ __forceinline__ void trace_point(const Item& it, const LensSmem& ls, uint64_t id, float zmin, float zmax,
                                            RayFwd& r) {
  r.iters = 0;
  float sx, sy, d0x, d0y, d0z, omc, sphi;
  source_ray(it, id, &sx, &sy, &d0x, &d0y, &d0z, &omc, &sphi);
  const float tau = (it.z_in - it.pz) * fast_rcp(d0z);
  const float ox = fmaf(tau, d0x, sx), oy = fmaf(tau, d0y, sy), oz = it.z_in;
  if (!(tau > 0.0f) || fabsf(ox) > it.rx || fabsf(oy) > it.ry) { r.status = FR_RAY_APERTURE_MISS; return; }
  // Snell air -> glass at the flat face, normal (0,0,1).
  const float eta1 = 1.0f / it.n_glass;
  r.dx = eta1 * d0x;
  r.dy = eta1 * d0y;
  r.dz = sqrtf(fmaf(-eta1 * eta1, sphi * sphi, 1.0f));
  const float om2 = omc * omc;
  r.T1 = (1.0f - it.R0) * fmaf(-om2 * om2, omc, 1.0f);
  exit_hit<MARCH>(it, ls, ox, oy, oz, zmin, zmax, r);
}

// ---------------------------------------------------------------------------
// Freeform entry face (both faces optimised, Sec. 4): the ray meets a second
// B-spline height field over the same aperture, refracts into the glass there,
// and the glass ray meets the exit freeform as a point-source ray does.
// ---------------------------------------------------------------------------
struct RayIn {
  int k, l;             // entry patch
  float s, t;           // patch coordinates of the entry point
  float ox, oy, oz;     // entry point
  float d0x, d0y, d0z;  // direction in air
  float Zs, Zt;         // entry slopes in patch coordinates
  float nx, ny, nz;     // entry normal, into the glass
  float invL;
  float c, cs, a;       // d0.n, transmitted cosine, c/n_glass - cs
  float tin, gpin;      // point source: ray parameter of the entry point, df_in/dt there
};

// f_in(t) = Z_in(o_uv + d_uv t) - o_z - d_z t on the entry net and df_in/dt.
__device__ __forceinline__ void f_eval_in(const Item& it, const LensSmem& li, float ou, float ov, float du, float dv,
                                          float oz, float dz, float t, RayIn& e, float* f, float* fp) {
  locate(fmaf(du, t, ou), it.nsu_in, &e.k, &e.s);
  locate(fmaf(dv, t, ov), it.nsv_in, &e.l, &e.t);
  float Z;
  patch_eval(li.patch + (size_t)(e.k * it.nsv_in + e.l) * 4, e.s, e.t, &Z, &e.Zs, &e.Zt);
  *f = Z - fmaf(dz, t, oz);
  *fp = fmaf(e.Zs, du * (float)it.nsu_in, fmaf(e.Zt, dv * (float)it.nsv_in, -dz));
}

// One ray through a two-face lens. Collimated rays (row, col) meet the entry
// face at (X(u), Y(v), Z_in(u,v)); point-source rays at the smallest root of
// f_in over the entry net's convex-hull slab, found by the same safeguarded
// Newton as the exit (the ray must be over the domain at the bottom of the slab
// and stay over it until the root: else it misses the aperture).
__device__ __forceinline__ void trace_two_face(const Item& it, const LensSmem& ls, const LensSmem& li, uint64_t id,
                                               uint32_t row, uint32_t col, RayFwd& r, RayIn& e) {
  r.iters = 0;
  if (it.kind == FR_SOURCE_COLLIMATED) {
    float ja = 0.5f, jb = 0.5f;
    if (it.jitter) {
      const uint2 w = philox_ray_words(it.seed, id);
      ja = unit23(w.x);
      jb = unit23(w.y);
    }
    const float u = ((float)col + ja) / (float)it.cols, v = ((float)row + jb) / (float)it.rows;
    e.d0x = 0.0f;
    e.d0y = 0.0f;
    e.d0z = 1.0f;
    locate(u, it.nsu_in, &e.k, &e.s);
    locate(v, it.nsv_in, &e.l, &e.t);
    float Z;
    patch_eval(li.patch + (size_t)(e.k * it.nsv_in + e.l) * 4, e.s, e.t, &Z, &e.Zs, &e.Zt);
    e.ox = fmaf(2.0f, u, -1.0f) * it.rx;
    e.oy = fmaf(2.0f, v, -1.0f) * it.ry;
    e.oz = Z;
  } else {
    float sx, sy, omc, sphi;
    source_ray(it, id, &sx, &sy, &e.d0x, &e.d0y, &e.d0z, &omc, &sphi);
    float zmin, zmax;
    zbounds(li, &zmin, &zmax);
    const float pad = 1e-6f * (1.0f + fmaxf(fabsf(zmin), fabsf(zmax)));
    const float inv_dz = fast_rcp(e.d0z);
    float ta = fmaxf(0.0f, (zmin - pad - it.pz) * inv_dz);
    const float t_hi = (zmax + pad - it.pz) * inv_dz;
    const float ou = fmaf(0.5f / it.rx, sx, 0.5f), ov = fmaf(0.5f / it.ry, sy, 0.5f);
    const float du = e.d0x * (0.5f / it.rx), dv = e.d0y * (0.5f / it.ry);
    const float ua = fmaf(du, ta, ou), va = fmaf(dv, ta, ov);
    if (!(ua >= 0.0f && ua <= 1.0f && va >= 0.0f && va <= 1.0f)) { r.status = FR_RAY_APERTURE_MISS; return; }
    float t_dom = INFINITY;
    if (du > 0.0f) t_dom = fminf(t_dom, (1.0f - ou) / du);
    if (du < 0.0f) t_dom = fminf(t_dom, -ou / du);
    if (dv > 0.0f) t_dom = fminf(t_dom, (1.0f - ov) / dv);
    if (dv < 0.0f) t_dom = fminf(t_dom, -ov / dv);
    const float tb = fminf(t_hi, t_dom);
    float f, fp;
    if (ta == 0.0f) {
      f_eval_in(it, li, ou, ov, du, dv, it.pz, e.d0z, 0.0f, e, &f, &fp);
      if (f < 0.0f) { r.status = FR_RAY_INVALID; return; }
    }
    // The smallest root, as for the exit face (first_root).
    const NetLine q{ou, ov, du, dv, it.pz, e.d0z};
    auto eval = [&](float t, float* fv, float* gv) { f_eval_in(it, li, ou, ov, du, dv, it.pz, e.d0z, t, e, fv, gv); };
    float t;
    int iters_in = 0;
    float gs, gt;
    slopes(li, &gs, &gt);
    const int found = first_root<true>(li.patch, li.hull, it.nsu_in, it.nsv_in, q, ta, tb, !(tb < t_hi), gs, gt,
                                       it.newton_max, it.newton_tol, eval, &t, &fp, &iters_in);
    if (found == ROOT_NONE) { r.status = FR_RAY_APERTURE_MISS; return; }   // leaves through the side first
    if (found == ROOT_FAIL) { r.status = FR_RAY_NEWTON_FAIL; return; }
    e.tin = t;
    e.gpin = fp;
    e.ox = fmaf(e.d0x, t, sx);
    e.oy = fmaf(e.d0y, t, sy);
    e.oz = fmaf(e.d0z, t, it.pz);
  }
  // Snell air -> glass at the entry normal (-Z_x, -Z_y, 1)/|.|; Schlick with
  // the incident cosine (in air).
  const float Zx = e.Zs * it.ku_in, Zy = e.Zt * it.kv_in;
  const float invL = rsqrtf(fmaf(Zx, Zx, fmaf(Zy, Zy, 1.0f)));
  e.invL = invL;
  e.nx = -Zx * invL;
  e.ny = -Zy * invL;
  e.nz = invL;
  const float c = fmaf(e.d0x, e.nx, fmaf(e.d0y, e.ny, e.d0z * e.nz));
  e.c = c;
  const float eta1 = 1.0f / it.n_glass;
  const float k = fmaf(-eta1 * eta1, fmaf(-c, c, 1.0f), 1.0f);   // > 0: into the denser medium
  e.cs = k * rsqrtf(k);
  e.a = fmaf(eta1, c, -e.cs);
  r.dx = fmaf(eta1, e.d0x, -e.a * e.nx);
  r.dy = fmaf(eta1, e.d0y, -e.a * e.ny);
  r.dz = fmaf(eta1, e.d0z, -e.a * e.nz);
  const float omc = 1.0f - c, om2 = omc * omc;
  r.T1 = (1.0f - it.R0) * fmaf(-om2 * om2, omc, 1.0f);
  float zmin, zmax;
  zbounds(ls, &zmin, &zmax);
  exit_hit<true>(it, ls, e.ox, e.oy, e.oz, zmin, zmax, r);
}

// ---------------------------------------------------------------------------
// Sec. 2.3: Gaussian reconstruction filter on the nu x nu footprint around the
// pixel that holds the hit; every other pixel has f = 0.
// ---------------------------------------------------------------------------
template <int NU>
struct Foot {
  int ie, je;           // extended column / row of the footprint's first cell
  float dx0, dy0;       // hit minus the centre of the first cell, in pixels
  float fx[NU], fy[NU]; // filter values
  float rsx, rsy;       // 1 / sum f
};

// Both axes at once: the x and y work of the filter runs as packed FP32 pairs
// (one add, multiply or FMA instruction for the two axes), except the
// exponentials, floors and clamps.
template <int NU>
__device__ __forceinline__ bool footprint(const Item& it, float X, float Y, Foot<NU>& f) {
  constexpr int h = (NU - 1) / 2;
  const float2 g = __ffma2_rn(make_float2(X, Y), make_float2(it.inv_wx, it.inv_wy), make_float2(it.gx_off, it.gy_off));
  const float flx = fminf(fmaxf(floorf(g.x), (float)h), (float)(it.nx + h - 1));
  const float fly = fminf(fmaxf(floorf(g.y), (float)h), (float)(it.ny + h - 1));
  f.ie = (int)flx - h;
  f.je = (int)fly - h;
  // g - (first + 0.5), in pixels, for each axis
  const float2 d0 = __fadd2_rn(__fadd2_rn(g, make_float2(-flx, -fly)), make_float2((float)h - 0.5f, (float)h - 0.5f));
  f.dx0 = d0.x;
  f.dy0 = d0.y;
  const float2 na = make_float2(-it.ax, -it.ay), ncut = make_float2(-it.cut, -it.cut);
  float2 sum = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    // Outside the support |d| >= nu/2 the exponential is at most `cut`, so the
    // clamp at 0 is the support test.
    const float2 d = __fadd2_rn(d0, make_float2(-(float)a, -(float)a));
    const float2 e = __fmul2_rn(__fmul2_rn(na, d), d);
    float2 v = __fadd2_rn(make_float2(ex2_approx(e.x), ex2_approx(e.y)), ncut);
    v.x = fmaxf(v.x, 0.0f);
    v.y = fmaxf(v.y, 0.0f);
    f.fx[a] = v.x;
    f.fy[a] = v.y;
    sum = __fadd2_rn(sum, v);
  }
  // For nu >= 3 the hit's own pixel is well inside the support: sum > 0.
  f.rsx = (NU >= 3 || sum.x > 0.0f) ? fast_rcp(sum.x) : 0.0f;
  f.rsy = (NU >= 3 || sum.y > 0.0f) ? fast_rcp(sum.y) : 0.0f;
  return NU >= 3 || (f.rsx > 0.0f && f.rsy > 0.0f);   // nu = 1 exactly on a pixel edge: all f = 0
}

template <int NU>
__device__ __forceinline__ void axis_footprint(float g, int n, float a2, float cut, int* first, float* d0, float* f,
                                               float* rs) {
  constexpr int h = (NU - 1) / 2;
  const float fl = fminf(fmaxf(floorf(g), (float)h), (float)(n + h - 1));
  *first = (int)fl - h;
  const float dfirst = g - fl + ((float)h - 0.5f);   // g - (first + 0.5)
  *d0 = dfirst;
  float sum = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    // Outside the support |d| >= nu/2 the exponential is at most `cut`, so the
    // clamp at 0 is the support test.
    const float d = dfirst - (float)a;
    f[a] = fmaxf(ex2_approx(-a2 * d * d) - cut, 0.0f);
    sum += f[a];
  }
  // For nu >= 3 the hit's own pixel is well inside the support: sum > 0.
  *rs = (NU >= 3 || sum > 0.0f) ? fast_rcp(sum) : 0.0f;
}

// The same footprint one axis at a time (the adjoint and tangent traces, whose
// register budget the packed pairs of `footprint` would strain); bit for bit
// the same values.
template <int NU>
__device__ __forceinline__ bool footprint_scalar(const Item& it, float X, float Y, Foot<NU>& f) {
  const float gx = fmaf(X, it.inv_wx, it.gx_off);
  const float gy = fmaf(Y, it.inv_wy, it.gy_off);
  axis_footprint<NU>(gx, it.nx, it.ax, it.cut, &f.ie, &f.dx0, f.fx, &f.rsx);
  axis_footprint<NU>(gy, it.ny, it.ay, it.cut, &f.je, &f.dy0, f.fy, &f.rsy);
  return NU >= 3 || (f.rsx > 0.0f && f.rsy > 0.0f);   // nu = 1 exactly on a pixel edge: all f = 0
}

// ---------------------------------------------------------------------------
// Lenses of degrees p, q from 1 to 5 (collimated sources only): the basis
// functions of each ray's span by the recursion, the heights in shared memory.
// ---------------------------------------------------------------------------
// Clamped uniform knot vector of degree p with ns non-empty spans:
// t_j = clamp((j - p) / ns, 0, 1).
__device__ __forceinline__ float knot_cu(int j, int p, int ns) {
  return fminf(fmaxf((float)(j - p) / (float)ns, 0.0f), 1.0f);
}

// The p + 1 basis functions of degree p (p <= 5) that are non-zero on the span
// of u, N_{k+a,p}(u) for a = 0..p, and their u-derivatives (Sec. 2.1): the
// Cox-de Boor recursion raised one degree at a time on the span's knots, and
// N'_{j,p} = p N_{j,p-1} / (t_{j+p} - t_j) - p N_{j+1,p-1} / (t_{j+p+1} - t_{j+1})
// from the degree p - 1 values. k: the span's first control index.
__device__ __forceinline__ void basis_general(int p, int ns, float u, int* k_out, float (&N)[6], float (&dN)[6]) {
  const int k = min((int)(u * (float)ns), ns - 1);
  const int i = k + p;   // the span is [t_i, t_{i+1})
  float left[6], right[6], M[6];
  N[0] = 1.0f;
  M[0] = 1.0f;
#pragma unroll 1
  for (int d = 1; d <= p; ++d) {
    left[d] = u - knot_cu(i + 1 - d, p, ns);
    right[d] = knot_cu(i + d, p, ns) - u;
    float saved = 0.0f;
#pragma unroll 1
    for (int r = 0; r < d; ++r) {
      const float den = right[r + 1] + left[d - r];
      const float tmp = den != 0.0f ? N[r] / den : 0.0f;
      N[r] = saved + right[r + 1] * tmp;
      saved = left[d - r] * tmp;
    }
    N[d] = saved;
    if (d == p - 1)
#pragma unroll 1
      for (int r = 0; r < p; ++r) M[r] = N[r];   // degree p - 1: N_{k+1+r,p-1}
  }
#pragma unroll 1
  for (int a = 0; a <= p; ++a) {
    float v = 0.0f;
    if (a >= 1) {
      const float den = knot_cu(i + a, p, ns) - knot_cu(i - p + a, p, ns);
      if (den != 0.0f) v += M[a - 1] / den;
    }
    if (a <= p - 1) {
      const float den = knot_cu(i + a + 1, p, ns) - knot_cu(i - p + a + 1, p, ns);
      if (den != 0.0f) v -= M[a] / den;
    }
    dN[a] = (float)p * v;
  }
  *k_out = k;
}

// Z and its u- and v-derivatives from a net in `P` (row-major, ncv columns).
__device__ __forceinline__ void surface_general(const float* P, int ncv, int k, int l, int p, int q,
                                                const float (&Nu)[6], const float (&dNu)[6], const float (&Nv)[6],
                                                const float (&dNv)[6], float* Z, float* Zu, float* Zv) {
  float z = 0.0f, zu = 0.0f, zv = 0.0f;
#pragma unroll 1
  for (int a = 0; a <= p; ++a) {
    float c = 0.0f, cv = 0.0f;
#pragma unroll 1
    for (int b = 0; b <= q; ++b) {
      const float w = P[(k + a) * ncv + l + b];
      c = fmaf(Nv[b], w, c);
      cv = fmaf(dNv[b], w, cv);
    }
    z = fmaf(Nu[a], c, z);
    zu = fmaf(dNu[a], c, zu);
    zv = fmaf(Nu[a], cv, zv);
  }
  *Z = z;
  *Zu = zu;
  *Zv = zv;
}

// Collimated ray `id` (cell centre or jittered) through a general-degree lens
// whose heights are in sP: its span (k, l), the basis functions and their
// u- and v-derivatives, and the traced ray. The slopes passed on are per unit
// of span coordinate (s = u nsu - k), as the bicubic kernels'.
__device__ __forceinline__ void trace_collimated_general(const Item& it, const float* sP, uint64_t id, float inv_cols,
                                                         float inv_rows, RayFwd& r, int* k, int* l, float (&Nu)[6],
                                                         float (&dNu)[6], float (&Nv)[6], float (&dNv)[6]) {
  const uint32_t row = (uint32_t)(id / (uint64_t)it.cols), col = (uint32_t)(id % (uint64_t)it.cols);
  float ja = 0.5f, jb = 0.5f;
  if (it.jitter) {
    const uint2 w = philox_ray_words(it.seed, id);
    ja = unit23(w.x);
    jb = unit23(w.y);
  }
  const float u = ((float)col + ja) * inv_cols, v = ((float)row + jb) * inv_rows;
  basis_general(it.p, it.nsu, u, k, Nu, dNu);
  basis_general(it.q, it.nsv, v, l, Nv, dNv);
  float Z, Zu, Zv;
  surface_general(sP, it.ncv, *k, *l, it.p, it.q, Nu, dNu, Nv, dNv, &Z, &Zu, &Zv);
  collimated_at(it, u, v, fmaf(2.0f, v, -1.0f) * it.ry, Z, Zu / (float)it.nsu, Zv / (float)it.nsv, r);
  r.k = *k;
  r.l = *l;
}

// Filter sizes 1 to 11 with the size a runtime value (the wide-filter traces,
// the general-degree derivative maps): the values of axis_footprint, in loops
// that are not unrolled.
constexpr int kWideNu = 11;
struct FootDyn {
  int ie, je;
  float dx0, dy0;
  float fx[kWideNu], fy[kWideNu];
  float rsx, rsy;
};

__device__ __forceinline__ void axis_footprint_dyn(float g, int n, int nu, float a2, float cut, int* first, float* d0,
                                                   float* f, float* rs) {
  const int h = (nu - 1) / 2;
  const float fl = fminf(fmaxf(floorf(g), (float)h), (float)(n + h - 1));
  *first = (int)fl - h;
  const float dfirst = g - fl + ((float)h - 0.5f);
  *d0 = dfirst;
  float sum = 0.0f;
#pragma unroll 1
  for (int a = 0; a < nu; ++a) {
    const float d = dfirst - (float)a;
    f[a] = fmaxf(ex2_approx(-a2 * d * d) - cut, 0.0f);
    sum += f[a];
  }
  *rs = sum > 0.0f ? fast_rcp(sum) : 0.0f;   // 0 only for nu = 1 exactly on a pixel edge
}

// False when the footprint is empty (nu = 1 exactly on a pixel edge).
__device__ __forceinline__ bool footprint_dyn(const Item& it, float X, float Y, FootDyn& f) {
  axis_footprint_dyn(fmaf(X, it.inv_wx, it.gx_off), it.nx, it.nu, it.ax, it.cut, &f.ie, &f.dx0, f.fx, &f.rsx);
  axis_footprint_dyn(fmaf(Y, it.inv_wy, it.gy_off), it.ny, it.nu, it.ay, it.cut, &f.je, &f.dy0, f.fy, &f.rsy);
  return f.rsx > 0.0f && f.rsy > 0.0f;
}

// filter_grad for a FootDyn: F = f / S and dF/dX (dF/dY) per axis.
__device__ __forceinline__ void filter_grad_dyn(const Item& it, const FootDyn& f, float* Fx, float* Fy, float* gxa,
                                                float* gya) {
  const float ln2 = 0.69314718055994531f;
  const float kx = -2.0f * (it.ax * ln2) * it.inv_wx, ky = -2.0f * (it.ay * ln2) * it.inv_wy;
  float Spx = 0.0f, Spy = 0.0f;
#pragma unroll 1
  for (int a = 0; a < it.nu; ++a) {
    const float gx = kx * (f.dx0 - (float)a) * (f.fx[a] + it.cut);
    const float gy = ky * (f.dy0 - (float)a) * (f.fy[a] + it.cut);
    gxa[a] = f.fx[a] != 0.0f ? gx : 0.0f;
    gya[a] = f.fy[a] != 0.0f ? gy : 0.0f;
    Spx += gxa[a];
    Spy += gya[a];
    Fx[a] = f.fx[a] * f.rsx;
    Fy[a] = f.fy[a] * f.rsy;
  }
#pragma unroll 1
  for (int a = 0; a < it.nu; ++a) {
    // nu = 1: the normalised filter is 1 on its pixel, its derivative 0
    gxa[a] = it.nu == 1 ? 0.0f : fmaf(-Fx[a], Spx, gxa[a]) * f.rsx;
    gya[a] = it.nu == 1 ? 0.0f : fmaf(-Fy[a], Spy, gya[a]) * f.rsy;
  }
}

// ---------------------------------------------------------------------------
// Reverse mode of one ray (a9). Input: G[b][a] = dL/dE on the footprint (row b,
// column a). Output: the adjoint zeta of the hit height and of the surface
// slopes, from which dL/dP^z_{k+a,l+b} = zeta N_a N_b + Zs_bar N'_a N_b
// + Zt_bar N_a N'_b.
// ---------------------------------------------------------------------------
// Normalised filter values on one footprint, F_a = f_a / S, and their
// derivatives with respect to the screen hit, dF_a/dX = (f'_a - F_a S') / S with
// f'_a = -2 alpha delta_a e_a / w. With nu = 1 the normalised filter is
// identically 1 on its pixel: dF = 0.
template <int NU>
__device__ __forceinline__ void filter_grad(const Item& it, const Foot<NU>& f, float (&Fx)[NU], float (&Fy)[NU],
                                            float (&gxa)[NU], float (&gya)[NU]) {
  // The x and y axes as packed FP32 pairs: each lane of a pair rounds as the
  // scalar operation would.
  const float ln2 = 0.69314718055994531f;
  const float2 k2 = make_float2(-2.0f * (it.ax * ln2) * it.inv_wx, -2.0f * (it.ay * ln2) * it.inv_wy);
  const float2 d0 = make_float2(f.dx0, f.dy0), rs = make_float2(f.rsx, f.rsy), cut = make_float2(it.cut, it.cut);
  float2 Sp = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    const float2 fa = make_float2(f.fx[a], f.fy[a]);
    const float2 d = __fadd2_rn(d0, make_float2(-(float)a, -(float)a));
    const float2 g = __fmul2_rn(__fmul2_rn(k2, d), __fadd2_rn(fa, cut));
    gxa[a] = f.fx[a] != 0.0f ? g.x : 0.0f;
    gya[a] = f.fy[a] != 0.0f ? g.y : 0.0f;
    Sp = __fadd2_rn(Sp, make_float2(gxa[a], gya[a]));
    const float2 F = __fmul2_rn(fa, rs);
    Fx[a] = F.x;
    Fy[a] = F.y;
  }
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    // (g - F S') / S, with the product fused as in the scalar form
    const float2 v = __fmul2_rn(__ffma2_rn(make_float2(-Fx[a], -Fy[a]), Sp, make_float2(gxa[a], gya[a])), rs);
    gxa[a] = NU == 1 ? 0.0f : v.x;
    gya[a] = NU == 1 ? 0.0f : v.y;
  }
}

template <bool COLL>
__device__ __forceinline__ void ray_reverse_tail(const Item& it, const LensSmem& ls, const RayFwd& r, float W,
                                                 float Xs, float Ys, float* zeta, float* Zs_bar, float* Zt_bar);

template <int NU, bool COLL>
__device__ __forceinline__ void ray_reverse(const Item& it, const LensSmem& ls, const RayFwd& r, const Foot<NU>& f,
                                            const float (&G)[NU][NU], float* zeta, float* Zs_bar, float* Zt_bar) {
  float Fx[NU], Fy[NU], gxa[NU], gya[NU];
  filter_grad<NU>(it, f, Fx, Fy, gxa, gya);
  // the footprint contractions, (A, B) and (wbar, Xs) as packed pairs
  float2 WX = make_float2(0.0f, 0.0f);
  float Ys = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    float2 AB = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < NU; ++b) AB = __ffma2_rn(make_float2(G[b][a], G[b][a]), make_float2(Fy[b], gya[b]), AB);
    WX = __ffma2_rn(make_float2(AB.x, AB.x), make_float2(Fx[a], gxa[a]), WX);
    Ys = fmaf(AB.y, Fx[a], Ys);
  }
  ray_reverse_tail<COLL>(it, ls, r, WX.x, WX.y, Ys, zeta, Zs_bar, Zt_bar);
}

// The chain of ray_reverse after the footprint contraction: from
// W = sum G F_x F_y, Xs = sum G F'_x F_y and Ys = sum G F_x F'_y to the
// adjoints of the hit height and slopes.
template <bool COLL>
__device__ __forceinline__ void ray_reverse_tail(const Item& it, const LensSmem& ls, const RayFwd& r, float W,
                                                 float Xs, float Ys, float* zeta, float* Zs_bar, float* Zt_bar) {
  float wbar = W;
  const float K = r.w * it.inv_area;
  wbar *= it.inv_area;
  const float2 XYbar = __fmul2_rn(make_float2(K, K), make_float2(Xs, Ys));
  const float Xbar = XYbar.x, Ybar = XYbar.y;
  // Propagation X = x + lam t_x, lam = (z_s - z)/t_z.
  const float2 txyb = __fmul2_rn(make_float2(r.lam, r.lam), XYbar);
  const float txb = txyb.x, tyb = txyb.y;
  const float lamb = fmaf(Xbar, r.tx, Ybar * r.ty);
  const float inv_tz = fast_rcp(r.tz);
  const float tzb = -lamb * r.lam * inv_tz;
  const float zbar = -lamb * inv_tz;
  // Weight w = omega0 T1 T2, T2 = (1-R0)(1-(1-cs)^5).
  const float om = 1.0f - r.cs;
  const float om2 = om * om;
  float csb = wbar * it.omega0 * r.T1 * (1.0f - it.R0) * 5.0f * om2 * om2;
  // Refraction t = eta d - a n, a = eta c - cs, cs = sqrt(1 - eta^2 (1 - c^2)), c = d.n.
  const float eta = it.n_glass;
  const float abar = -(txb * r.nx + tyb * r.ny + tzb * r.nz);
  float nbx = -r.a * txb, nby = -r.a * tyb, nbz = -r.a * tzb;
  float cbar = eta * abar;
  csb -= abar;
  const float kbar = csb * 0.5f * fast_rcp(r.cs);
  cbar = fmaf(kbar * 2.0f * eta * eta, r.c, cbar);
  if (COLL) {
    nbz += cbar;
  } else {
    nbx = fmaf(cbar, r.dx, nbx);
    nby = fmaf(cbar, r.dy, nby);
    nbz = fmaf(cbar, r.dz, nbz);
  }
  // Normalisation n = m / |m|, m = (-Z_x, -Z_y, 1).
  const float ndot = nbx * r.nx + nby * r.ny + nbz * r.nz;
  const float mbx = (nbx - ndot * r.nx) * r.invL;
  const float mby = (nby - ndot * r.ny) * r.invL;
  *Zs_bar = -mbx * it.ku;
  *Zt_bar = -mby * it.kv;
  if (COLL) {
    *zeta = zbar;   // the hit height is Z itself
    return;
  }
  // Point source: the hit moves along the ray with t*; the implicit function
  // theorem on f(t*, P) = 0 gives dt*/dP_ab = -N_a N_b / f'(t*).
  float Zss, Zst, Ztt;
  patch_eval2(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Zss, &Zst, &Ztt);
  const float dsdt = r.dx * (0.5f / it.rx) * (float)it.nsu;
  const float dtdt = r.dy * (0.5f / it.ry) * (float)it.nsv;
  const float tbar = Xbar * r.dx + Ybar * r.dy + zbar * r.dz +
                     *Zs_bar * fmaf(Zss, dsdt, Zst * dtdt) + *Zt_bar * fmaf(Zst, dsdt, Ztt * dtdt);
  *zeta = -tbar / r.gp;
}

// ---------------------------------------------------------------------------
// Forward mode of one ray (Sec. 3.1 derivative maps): the tangents of the screen
// hit and of the weight for a tangent of the freeform hit (hx, hy, hz) and of
// its slopes in patch coordinates (dZs, dZt), through the exit refraction,
// Schlick and the propagation. Transposes the chain of ray_reverse.
// ---------------------------------------------------------------------------
struct RayTan {
  float dX, dY, dw;
};

template <bool COLL>
__device__ __forceinline__ RayTan ray_tangent(const Item& it, const RayFwd& r, float hx, float hy, float hz,
                                              float dZs, float dZt) {
  // n = m / |m|, m = (-Z_x, -Z_y, 1): dn = (dm - n (n.dm)) / |m|.
  const float dZx = dZs * it.ku, dZy = dZt * it.kv;
  const float ndm = -fmaf(r.nx, dZx, r.ny * dZy);
  const float dnx = fmaf(-r.nx, ndm, -dZx) * r.invL;
  const float dny = fmaf(-r.ny, ndm, -dZy) * r.invL;
  const float dnz = -r.nz * ndm * r.invL;
  // c = d.n, cs = sqrt(1 - eta^2 (1 - c^2)), a = eta c - cs, t = eta d - a n.
  const float dc = COLL ? dnz : fmaf(r.dx, dnx, fmaf(r.dy, dny, r.dz * dnz));
  const float eta = it.n_glass;
  const float dcs = eta * eta * r.c * dc * fast_rcp(r.cs);
  const float da = fmaf(eta, dc, -dcs);
  const float dtx = fmaf(-da, r.nx, -r.a * dnx);
  const float dty = fmaf(-da, r.ny, -r.a * dny);
  const float dtz = fmaf(-da, r.nz, -r.a * dnz);
  // w = omega0 T1 T2, T2 = (1-R0)(1-(1-cs)^5).
  const float om = 1.0f - r.cs;
  const float om2 = om * om;
  RayTan o;
  o.dw = it.omega0 * r.T1 * (1.0f - it.R0) * 5.0f * om2 * om2 * dcs;
  // X = x + lam t_x, lam = (z_s - z) / t_z.
  const float dlam = -fmaf(r.lam, dtz, hz) * fast_rcp(r.tz);
  o.dX = fmaf(dlam, r.tx, fmaf(r.lam, dtx, hx));
  o.dY = fmaf(dlam, r.ty, fmaf(r.lam, dty, hy));
  return o;
}

// Reverse mode of one ray through a two-face lens: the exit net's adjoints
// (zeta, Zs_bar, Zt_bar at the exit hit, as ray_reverse) and the entry net's
// (zeta_in, Zs_bar_in, Zt_bar_in at the entry point). The glass ray's origin o
// and direction d now depend on the entry net: their adjoints gather from the
// exit refraction, the exit hit h = o + d t* and the implicit function theorem
// on f(t*; o, d, P) = 0 (df/do = (Z_x, Z_y, -1), df/dd = t* df/do), and go back
// through Snell at the entry face (with Schlick's T1 of the incident cosine),
// the entry normal and the entry point (for a point source, its own implicit
// function theorem on f_in).
template <int NU>
__device__ __forceinline__ void ray_reverse_two(const Item& it, const LensSmem& ls, const LensSmem& li, const RayFwd& r,
                                                const RayIn& e, const Foot<NU>& f, const float (&G)[NU][NU],
                                                float* zeta, float* Zs_bar, float* Zt_bar, float* zeta_in,
                                                float* Zs_bar_in, float* Zt_bar_in) {
  float Fx[NU], Fy[NU], gxa[NU], gya[NU];
  filter_grad<NU>(it, f, Fx, Fy, gxa, gya);
  float wbar = 0.0f, Xs = 0.0f, Ys = 0.0f;
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    float A = 0.0f, B = 0.0f;
#pragma unroll
    for (int b = 0; b < NU; ++b) {
      A = fmaf(G[b][a], Fy[b], A);
      B = fmaf(G[b][a], gya[b], B);
    }
    wbar = fmaf(A, Fx[a], wbar);
    Xs = fmaf(A, gxa[a], Xs);
    Ys = fmaf(B, Fx[a], Ys);
  }
  const float K = r.w * it.inv_area;
  wbar *= it.inv_area;
  const float Xbar = K * Xs, Ybar = K * Ys;
  // Propagation X = h + lam t, lam = (z_s - h_z)/t_z.
  const float txb = r.lam * Xbar, tyb = r.lam * Ybar;
  const float lamb = fmaf(Xbar, r.tx, Ybar * r.ty);
  const float inv_tz = fast_rcp(r.tz);
  const float tzb = -lamb * r.lam * inv_tz;
  const float hzb0 = -lamb * inv_tz;
  // Weight w = omega0 T1 T2.
  const float om = 1.0f - r.cs, om2 = om * om;
  float csb = wbar * it.omega0 * r.T1 * (1.0f - it.R0) * 5.0f * om2 * om2;
  const float T1b = wbar * it.omega0 * r.T2;
  // Exit refraction t = eta d - a n, a = eta c - cs, c = d.n.
  const float eta = it.n_glass;
  const float abar = -(txb * r.nx + tyb * r.ny + tzb * r.nz);
  float nbx = -r.a * txb, nby = -r.a * tyb, nbz = -r.a * tzb;
  float dbx = eta * txb, dby = eta * tyb, dbz = eta * tzb;
  float cbar = eta * abar;
  csb -= abar;
  cbar = fmaf(csb * eta * eta * r.c, fast_rcp(r.cs), cbar);
  nbx = fmaf(cbar, r.dx, nbx);
  nby = fmaf(cbar, r.dy, nby);
  nbz = fmaf(cbar, r.dz, nbz);
  dbx = fmaf(cbar, r.nx, dbx);
  dby = fmaf(cbar, r.ny, dby);
  dbz = fmaf(cbar, r.nz, dbz);
  // Exit normal n = m/|m|, m = (-Z_x, -Z_y, 1).
  const float ndot = nbx * r.nx + nby * r.ny + nbz * r.nz;
  const float zsb = -((nbx - ndot * r.nx) * r.invL) * it.ku;
  const float ztb = -((nby - ndot * r.ny) * r.invL) * it.kv;
  *Zs_bar = zsb;
  *Zt_bar = ztb;
  // Exit hit h = o + d t*; the slopes are taken at h.
  float Zss, Zst, Ztt;
  patch_eval2(ls.patch + (size_t)(r.k * it.nsv + r.l) * 4, r.s, r.t, &Zss, &Zst, &Ztt);
  const float hbx = fmaf(it.ku, fmaf(zsb, Zss, ztb * Zst), Xbar);
  const float hby = fmaf(it.kv, fmaf(zsb, Zst, ztb * Ztt), Ybar);
  const float hbz = hzb0;
  const float tbar = fmaf(hbx, r.dx, fmaf(hby, r.dy, hbz * r.dz));
  const float z = -tbar / r.gp;
  *zeta = z;
  const float fx = r.Zs * it.ku, fy = r.Zt * it.kv;
  float obx = fmaf(z, fx, hbx), oby = fmaf(z, fy, hby), obz = hbz - z;
  const float zt = z * r.tstar;
  dbx = fmaf(hbx, r.tstar, fmaf(zt, fx, dbx));
  dby = fmaf(hby, r.tstar, fmaf(zt, fy, dby));
  dbz = fmaf(hbz, r.tstar, fmaf(-zt, 1.0f, dbz));
  // Entry refraction d = eta1 d0 - a1 m, a1 = eta1 c1 - cs1, c1 = d0.m; T1(c1).
  const float eta1 = 1.0f / it.n_glass;
  const float a1b = -(dbx * e.nx + dby * e.ny + dbz * e.nz);
  float mbx = -e.a * dbx, mby = -e.a * dby, mbz = -e.a * dbz;
  float c1b = eta1 * a1b;
  c1b = fmaf(-a1b * eta1 * eta1 * e.c, fast_rcp(e.cs), c1b);
  const float om1 = 1.0f - e.c, om1_2 = om1 * om1;
  c1b = fmaf(T1b * (1.0f - it.R0) * 5.0f, om1_2 * om1_2, c1b);
  mbx = fmaf(c1b, e.d0x, mbx);
  mby = fmaf(c1b, e.d0y, mby);
  mbz = fmaf(c1b, e.d0z, mbz);
  // Entry normal.
  const float nd = mbx * e.nx + mby * e.ny + mbz * e.nz;
  const float zsbi = -((mbx - nd * e.nx) * e.invL) * it.ku_in;
  const float ztbi = -((mby - nd * e.ny) * e.invL) * it.kv_in;
  *Zs_bar_in = zsbi;
  *Zt_bar_in = ztbi;
  if (it.kind == FR_SOURCE_COLLIMATED) {
    *zeta_in = obz;   // the entry point's height at a fixed (u, v)
    return;
  }
  // Point source: the entry point moves along the source ray with t_in.
  float Sss, Sst, Stt;
  patch_eval2(li.patch + (size_t)(e.k * it.nsv_in + e.l) * 4, e.s, e.t, &Sss, &Sst, &Stt);
  obx = fmaf(it.ku_in, fmaf(zsbi, Sss, ztbi * Sst), obx);
  oby = fmaf(it.kv_in, fmaf(zsbi, Sst, ztbi * Stt), oby);
  const float tinb = fmaf(obx, e.d0x, fmaf(oby, e.d0y, obz * e.d0z));
  *zeta_in = -tinb / e.gpin;
}

// Ray counts by cause (FR_RAY_*): a per-thread count of deposited rays and
// shared-memory counters for the rest (only when the caller asked for them).
struct RayCount {
  unsigned int on_screen;
  __device__ __forceinline__ void add(int status, unsigned int* s_cnt) {
    if (status == FR_RAY_ON_SCREEN) ++on_screen;
    else if (s_cnt) atomicAdd(&s_cnt[status], 1u);
  }
  // All lanes of every warp call this.
  __device__ __forceinline__ void reduce_into(unsigned int* s_cnt) const {
    const unsigned int v = __reduce_add_sync(0xffffffffu, on_screen);
    if ((threadIdx.x & 31) == 0 && v && s_cnt) atomicAdd(&s_cnt[FR_RAY_ON_SCREEN], v);
  }
  // After a __syncthreads that follows reduce_into.
  static __device__ __forceinline__ void publish(const unsigned int* s_cnt, fr_stats* stats) {
    if (stats && threadIdx.x < FR_RAY_NCAUSES && s_cnt[threadIdx.x])
      atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rays[threadIdx.x]),
                (unsigned long long)s_cnt[threadIdx.x]);
  }
};

// With a ray order (fr_ray_order): the number H of rays that meet the aperture,
// stored after the permutation; they fill its positions 0..H-1, the others
// miss the aperture.
__device__ __forceinline__ uint64_t ordered_hits(const Item& it) {
  return min((uint64_t)__ldg(it.order + it.n_rays), it.n_rays);
}

// The rays [a, b) of this lane: the item's rays are split evenly over all warps
// of the item's CTAs, and each warp's share evenly over its 32 lanes, so every
// lane traces a run of consecutive ray ids (consecutive grid cells of one row
// for a collimated source). With a ray order the positions 0..H-1 are split:
// the rays that miss the aperture are only counted (ordered_misses_into).
__device__ __forceinline__ void lane_range(const Item& it, int warps, uint64_t* a, uint64_t* b) {
  const uint64_t lo = it.order ? 0 : it.ray_begin;
  const uint64_t n = it.order ? ordered_hits(it) : it.ray_end - it.ray_begin;
  const uint64_t W = (uint64_t)(it.cta_end - it.cta_begin) * (uint64_t)warps;
  const uint64_t gw = (uint64_t)((int)blockIdx.x - it.cta_begin) * (uint64_t)warps + (threadIdx.x >> 5);
  const uint64_t w0 = n * gw / W, w1 = n * (gw + 1) / W;
  const uint64_t m = w1 - w0, lane = threadIdx.x & 31;
  *a = lo + w0 + m * lane / 32;
  *b = lo + w0 + m * (lane + 1) / 32;
}

// With a ray order the traces split the positions into chunks of kOrderChunk
// consecutive positions (a chunk is coherent: one cell of one knot span,
// neighbouring pixels). The float-mode point traces (k_forward, k_adjoint)
// take groups of 32 neighbouring chunks, one per lane, warp by warp from a
// per-CTA counter, the CTAs owning the groups in turn: the lanes of a warp
// then share a patch (broadcast table reads, agreeing Newton iterations) and
// the warps of a CTA finish together. OrderCursor deals the chunks statically
// for the other kernels: `near` gives the lanes of a warp neighbouring
// chunks, `spread` chunks far apart (the fixed-point adjoint, whose gradient
// flushes then go to different addresses). On the 16M-ray point source the
// counter took the forward from 475 to 438 us, chunks of 8 instead of 16 and
// the order's cells on the plane of the mean height to 429 us; the adjoint
// went from 1031 us (`spread`) to 999 us (counter) and 696 us (cells on that
// plane: the knot span of the hit changes once per 30 positions of the order
// instead of once per 10, and each change costs a lane a flush of its 16
// register sums).
constexpr uint64_t kOrderChunk = 8;

struct OrderCursor {
  uint64_t p, hi, c, lanes, H;
  __device__ __forceinline__ void init(const Item& it, bool spread) {
    const uint64_t warps = blockDim.x >> 5;
    const uint64_t Wt = (uint64_t)(it.cta_end - it.cta_begin) * warps;   // warps of the item
    const uint64_t gw = (uint64_t)((int)blockIdx.x - it.cta_begin) * warps + (threadIdx.x >> 5);
    const uint64_t lane = threadIdx.x & 31;
    H = ordered_hits(it);
    lanes = Wt * 32;
    // first chunk: near, lane L of warp gw takes 32 gw + L; spread, L Wt + gw
    c = spread ? lane * Wt + gw : gw * 32 + lane;
    start();
  }
  __device__ __forceinline__ void start() {
    p = c * kOrderChunk;
    hi = min(p + kOrderChunk, H);
    if (p >= H) p = hi = H;
  }
  __device__ __forceinline__ bool valid() const { return p < hi; }
  __device__ __forceinline__ void advance() {
    if (++p == hi) {
      c += lanes;
      start();
    }
  }
  // Most positions one CTA of `warps` warps can take (for fixed-point bounds);
  // also a bound for the traces that deal groups of 32 chunks to the CTAs in
  // turn (at most warps x that many chunks each).
  static __device__ __forceinline__ uint64_t max_per_cta(const Item& it, int warps) {
    const uint64_t lanes = (uint64_t)(it.cta_end - it.cta_begin) * (uint64_t)warps * 32;
    const uint64_t chunks = (ordered_hits(it) + kOrderChunk - 1) / kOrderChunk;
    return (chunks + lanes - 1) / lanes * kOrderChunk * (uint64_t)warps * 32;
  }
};

// Appends ray `id` of a hot trace kernel to the item's deferred list.
__device__ __forceinline__ void defer_ray(const Item& it, uint64_t id) {
  const uint32_t slot = atomicAdd(it.defer_n, 1u);
  it.defer[slot] = (uint32_t)(id - it.ray_begin);
}

// One thread of the item's first CTA adds the ordered aperture misses to the
// CTA's cause counters (s_cnt may be null: no counts asked for).
__device__ __forceinline__ void ordered_misses_into(const Item& it, unsigned int* s_cnt) {
  if (it.order && s_cnt && (int)blockIdx.x == it.cta_begin && threadIdx.x == 0)
    atomicAdd(&s_cnt[FR_RAY_APERTURE_MISS], (unsigned int)(it.n_rays - ordered_hits(it)));
}

}  // namespace fr
