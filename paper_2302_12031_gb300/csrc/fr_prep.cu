// Prep kernel: per lens, the power form of the bicubic B-spline on every knot
// span (Sec. 2.1) and the convex-hull bounds of the height field (Sec. 2.1.2).
//
// On span k of a clamped uniform knot vector the four non-zero basis functions
// N_{k..k+3,3} are cubics in the local coordinate s = u*nspan - k. Running the
// Cox-de Boor recursion on polynomials in s gives their coefficients exactly
// (up to rounding); the surface on span product (k, l) is then
//   Z(s,t) = sum_{a,b} N_{k+a}(s) N_{l+b}(t) P^z_{k+a,l+b} = sum_{e,f} C[e][f] s^e t^f.
#include "fr_internal.h"

namespace fr {
namespace {

// Clamped uniform knot u_j for n+1 control points of degree 3 (n+5 knots).
__device__ double knot(int j, int nspan) {
  const double u = (double)(j - 3) / (double)nspan;
  return u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
}

// Coefficients (in powers of s) of N_{k+a,3} on span k, a = 0..3.
__device__ void span_basis(int k, int nspan, double out[4][4]) {
  const int i = k + 3;                       // knot index of the span's left end
  const double h = 1.0 / (double)nspan;
  const double ui = knot(i, nspan);
  // poly[j - (i-3)][e]: coefficient of s^e of N_{j,d} restricted to the span.
  double poly[5][4] = {};
  poly[3][0] = 1.0;                          // N_{i,0} = 1 on its own span
  for (int d = 1; d <= 3; ++d) {
    double next[5][4] = {};
    for (int j = i - d; j <= i; ++j) {
      const int jj = j - (i - 3);
      const double den1 = knot(j + d, nspan) - knot(j, nspan);
      const double den2 = knot(j + d + 1, nspan) - knot(j + 1, nspan);
      for (int e = 3; e >= 0; --e) {
        double c = 0.0;
        if (den1 != 0.0) {
          // (u - u_j)/den1 * N_{j,d-1}, u - u_j = (ui - u_j) + h s
          const double c0 = (ui - knot(j, nspan)) / den1, c1 = h / den1;
          c += c0 * poly[jj][e] + (e > 0 ? c1 * poly[jj][e - 1] : 0.0);
        }
        if (den2 != 0.0 && jj + 1 <= 4) {
          // (u_{j+d+1} - u)/den2 * N_{j+1,d-1}, u_{j+d+1} - u = (u_{j+d+1} - ui) - h s
          const double c0 = (knot(j + d + 1, nspan) - ui) / den2, c1 = -h / den2;
          c += c0 * poly[jj + 1][e] + (e > 0 ? c1 * poly[jj + 1][e - 1] : 0.0);
        }
        next[jj][e] = c;
      }
    }
    for (int a = 0; a < 5; ++a)
      for (int e = 0; e < 4; ++e) poly[a][e] = next[a][e];
  }
  for (int a = 0; a < 4; ++a)
    for (int e = 0; e < 4; ++e) out[a][e] = poly[a][e];
}

__global__ void k_prep(const __grid_constant__ Launch<kMaxItems> L) {
  const Item& it = L.items[blockIdx.x];
  __shared__ float4 bu[kMaxSpans * 4], bv[kMaxSpans * 4];
  __shared__ float red_min[32], red_max[32];
  // Basis tables.
  for (int k = threadIdx.x; k < it.nsu + it.nsv; k += blockDim.x) {
    const bool isu = k < it.nsu;
    const int kk = isu ? k : k - it.nsu;
    double B[4][4];
    span_basis(kk, isu ? it.nsu : it.nsv, B);
    float4* dst = isu ? bu : bv;
    float4* gdst = isu ? it.basis_u : it.basis_v;
    for (int a = 0; a < 4; ++a) {
      const float4 q = make_float4((float)B[a][0], (float)B[a][1], (float)B[a][2], (float)B[a][3]);
      dst[kk * 4 + a] = q;
      gdst[kk * 4 + a] = q;
    }
  }
  __syncthreads();
  // Patches: C[e][f] = sum_a sum_b Bu[a][e] Bv[b][f] P[k+a][l+b].
  const int npatch = it.nsu * it.nsv;
  for (int pidx = threadIdx.x; pidx < npatch; pidx += blockDim.x) {
    const int k = pidx / it.nsv, l = pidx - k * it.nsv;
    float T[4][4];  // T[a][f] = sum_b P[k+a][l+b] Bv[b][f]
    for (int a = 0; a < 4; ++a) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int b = 0; b < 4; ++b) {
        const float Pab = it.ctrl[(k + a) * it.ncv + (l + b)];
        const float4 q = bv[l * 4 + b];
        acc[0] = fmaf(Pab, q.x, acc[0]);
        acc[1] = fmaf(Pab, q.y, acc[1]);
        acc[2] = fmaf(Pab, q.z, acc[2]);
        acc[3] = fmaf(Pab, q.w, acc[3]);
      }
      for (int f = 0; f < 4; ++f) T[a][f] = acc[f];
    }
    float4* out = it.patch + (size_t)pidx * 4;
    for (int e = 0; e < 4; ++e) {
      float c[4];
      for (int f = 0; f < 4; ++f) {
        float acc = 0.0f;
        for (int a = 0; a < 4; ++a) {
          const float4 q = bu[k * 4 + a];
          const float be = e == 0 ? q.x : (e == 1 ? q.y : (e == 2 ? q.z : q.w));
          acc = fmaf(be, T[a][f], acc);
        }
        c[f] = acc;
      }
      out[e] = make_float4(c[0], c[1], c[2], c[3]);
    }
  }
  // Convex hull of the control heights.
  float zmn = INFINITY, zmx = -INFINITY;
  for (int q = threadIdx.x; q < it.ncu * it.ncv; q += blockDim.x) {
    const float z = it.ctrl[q];
    zmn = fminf(zmn, z);
    zmx = fmaxf(zmx, z);
  }
  for (int o = 16; o > 0; o >>= 1) {
    zmn = fminf(zmn, __shfl_xor_sync(0xffffffffu, zmn, o));
    zmx = fmaxf(zmx, __shfl_xor_sync(0xffffffffu, zmx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_min[threadIdx.x >> 5] = zmn;
    red_max[threadIdx.x >> 5] = zmx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      zmn = fminf(zmn, red_min[w]);
      zmx = fmaxf(zmx, red_max[w]);
    }
    it.zb[0] = zmn;
    it.zb[1] = zmx;
  }
}

}  // namespace

cudaError_t launch_prep(const Item* items, int n_items, cudaStream_t st) {
  Launch<kMaxItems> L{};
  L.n_items = n_items;
  for (int i = 0; i < n_items; ++i) L.items[i] = items[i];
  k_prep<<<n_items, 256, 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace fr
