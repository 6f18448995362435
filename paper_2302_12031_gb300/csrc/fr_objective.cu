// The objective and parametrisation around the trace:
//  - the squared L2 loss (row a8) and the paper's normalised Frobenius loss
//    (Sec. 2.5, Eq. pipelineLoss) with their gradients, each one launch of one
//    thread-block cluster whose CTAs reduce through distributed shared memory
//    in a fixed order (bit-identical run to run, no atomics, no counters, no
//    scratch memory);
//  - control heights from unconstrained variables through tanh onto
//    (z_min, z_max) plus an offset f(P^x, P^y) (Sec. 2.4.2, Eqs. outputcorrection
//    and outputcorrectionwfunc), its adjoint, the spherical offsets of Table
//    magndata at the Greville points (Sec. 2.1), and Adam on the unconstrained
//    variables fused with both maps.
#include <cooperative_groups.h>

#include "fr_device.cuh"

namespace cg = cooperative_groups;

namespace fr {
namespace {

constexpr int kObjCluster = 8;      // CTAs of the loss cluster (portable cluster size)
constexpr int kObjThreads = 1024;
constexpr int kObjUnroll = 4;       // loads in flight per thread and loop trip

// FP64 runs at a small fraction of the FP32 rate on this GPU, so the sums below
// take each thread's FP32 partial sum through an FP32 xor tree within the warp
// and only then go to FP64: one warp adds the warps' sums, one thread per CTA
// adds the CTAs' sums in rank order through distributed shared memory. The
// order is fixed: the totals are bit-identical run to run. On return s_tot
// holds the totals (valid after the __syncthreads at the end). s_cta is this
// call's own slot: the other CTAs read it after the cluster barrier, so a later
// call must use another, and the kernel must pass one more cluster barrier
// before it exits.
template <int NV>
__device__ __forceinline__ void cluster_sum(const float (&v)[NV], double* s_warp, double* s_cta, double* s_tot) {
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) s_warp[warp * NV + k] = (double)x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < (int)(blockDim.x >> 5) ? s_warp[lane * NV + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) s_cta[k] = x;
    }
  }
  cl.sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (unsigned r = 0; r < cl.num_blocks(); ++r) t += *cl.map_shared_rank(s_cta + k, r);
      s_tot[k] = t;
    }
  }
  __syncthreads();
}

// A product e * r with r = rh + rl (two floats), kept as the unevaluated sum
// hi + lo: hi = e rh rounded, lo = its rounding error (exact by FMA) + e rl.
// About 2^-44 relative: the difference of two such products keeps its
// precision where they nearly cancel. Explicit _rn intrinsics: no contraction,
// so the same inputs give the same bits wherever this is evaluated.
__device__ __forceinline__ void mul_df(float e, float rh, float rl, float* hi, float* lo) {
  const float h = __fmul_rn(e, rh);
  *hi = h;
  *lo = __fmaf_rn(e, rl, __fmaf_rn(e, rh, -h));
}

// 1/S as a pair of floats rh + rl.
__device__ __forceinline__ void recip_df(double S, float* rh, float* rl) {
  const double r = 1.0 / S;
  *rh = (float)r;
  *rl = (float)(r - (double)*rh);
}

// D = E/S - E_ref/S_ref from the two products; *I = E/S (its leading float).
__device__ __forceinline__ float diff_df(float e, float er, const float* sc, float* I) {
  float Ih, Il, Rh, Rl;
  mul_df(e, sc[0], sc[1], &Ih, &Il);
  mul_df(er, sc[2], sc[3], &Rh, &Rl);
  *I = Ih;
  return __fadd_rn(__fsub_rn(Ih, Rh), __fsub_rn(Il, Rl));
}

// Interior pixel k (row-major over ny x nx) -> its cell on the extended grid.
__device__ __forceinline__ int ext_cell(int k, int nx, int hx, int hy, int ncol) {
  const int j = k / nx, i = k - j * nx;
  return (j + hy) * ncol + (i + hx);
}

// With I^ = E/S, I^_ref = E_ref/S_ref over the interior and D = I^ - I^_ref:
// L = ||D||_F / sqrt(nx ny), and dL/dE = (c D - c sum(D I^)) / S on the interior
// with c = 1/(sqrt(nx ny) ||D||_F), 0 on ghost pixels. ||D|| = 0 gives a zero
// gradient; S <= 0 or S_ref <= 0 gives L = NaN and a zero gradient.
// Per pixel the work is FP32, with D in the paired form above; images equal up
// to a power-of-two scale give D = 0 exactly (every step scales exactly).
__global__ void __cluster_dims__(kObjCluster, 1, 1) __launch_bounds__(kObjThreads)
    k_loss_frobenius(const float* __restrict__ E, const float* __restrict__ Eref, int nx, int ny, int hx, int hy,
                     int ncol, int nrow, double* __restrict__ loss, float* __restrict__ dLdE) {
  __shared__ double s_warp[(kObjThreads / 32) * 2];
  __shared__ double s_sums[2], s_dots[2], s_tot[2];
  __shared__ float s_sc[6];          // 1/S and 1/S_ref as float pairs, c, c sum(D I^)
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = kObjCluster * kObjThreads;
  const int tid = (int)cl.block_rank() * kObjThreads + threadIdx.x;
  const int n = nx * ny;
  pdl_trigger();
  pdl_wait();      // E is the previous kernel's output

  float p[2] = {0.0f, 0.0f};
  for (int k0 = tid; k0 < n; k0 += kObjUnroll * nthr) {
    float e[kObjUnroll], r[kObjUnroll];
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int k = k0 + u * nthr;
      e[u] = k < n ? E[ext_cell(k, nx, hx, hy, ncol)] : 0.0f;
      r[u] = k < n ? Eref[k] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      p[0] = __fadd_rn(p[0], e[u]);
      p[1] = __fadd_rn(p[1], r[u]);
    }
  }
  cluster_sum<2>(p, s_warp, s_sums, s_tot);
  const bool ok = s_tot[0] > 0.0 && s_tot[1] > 0.0;
  if (threadIdx.x == 0) {
    s_sc[0] = s_sc[1] = s_sc[2] = s_sc[3] = 0.0f;
    if (ok) {
      recip_df(s_tot[0], &s_sc[0], &s_sc[1]);
      recip_df(s_tot[1], &s_sc[2], &s_sc[3]);
    }
  }
  __syncthreads();
  const float sc[4] = {s_sc[0], s_sc[1], s_sc[2], s_sc[3]};

  float d[2] = {0.0f, 0.0f};         // sum D^2, sum D I^
  for (int k0 = tid; k0 < n; k0 += kObjUnroll * nthr) {
    float e[kObjUnroll], r[kObjUnroll];
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int k = k0 + u * nthr;
      e[u] = k < n ? E[ext_cell(k, nx, hx, hy, ncol)] : 0.0f;
      r[u] = k < n ? Eref[k] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      float I;
      const float D = diff_df(e[u], r[u], sc, &I);    // 0 for the padding (e = r = 0)
      d[0] = __fmaf_rn(D, D, d[0]);
      d[1] = __fmaf_rn(D, I, d[1]);
    }
  }
  cluster_sum<2>(d, s_warp, s_dots, s_tot);
  if (threadIdx.x == 0) {
    const double root_n = sqrt((double)nx * (double)ny);
    const double norm = sqrt(s_tot[0]);
    const double c = (ok && norm > 0.0) ? 1.0 / (root_n * norm) : 0.0;
    s_sc[4] = (float)c;
    s_sc[5] = (float)(c * s_tot[1]);
    if (cl.block_rank() == 0) *loss = ok ? norm / root_n : __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  const float cf = s_sc[4], gdot = s_sc[5];

  const int ncell = ncol * nrow;
  for (int q0 = tid; q0 < ncell; q0 += kObjUnroll * nthr) {
    float e[kObjUnroll], r[kObjUnroll];
    bool in[kObjUnroll];
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int q = q0 + u * nthr;
      const int row = q / ncol, col = q - row * ncol;
      const int i = col - hx, j = row - hy;
      in[u] = q < ncell && cf != 0.0f && i >= 0 && i < nx && j >= 0 && j < ny;
      e[u] = in[u] ? E[q] : 0.0f;
      r[u] = in[u] ? Eref[(size_t)j * nx + i] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int q = q0 + u * nthr;
      if (q >= ncell) break;
      float I;
      const float D = diff_df(e[u], r[u], sc, &I);
      dLdE[q] = in[u] ? __fmaf_rn(cf, D, -gdot) * sc[0] : 0.0f;
    }
  }
  cl.sync();       // no CTA leaves while another may still read its shared memory
}

// Squared L2 loss (row a8): L = sum over the interior of (E - E_ref)^2 and
// dL/dE = 2 (E - E_ref) there, 0 on ghost pixels; one pass, FP32 per pixel,
// the partial sums reduced over the cluster in a fixed order.
__global__ void __cluster_dims__(kObjCluster, 1, 1) __launch_bounds__(kObjThreads)
    k_loss_l2(const float* __restrict__ E, const float* __restrict__ Eref, int nx, int ny, int hx, int hy, int ncol,
              int nrow, double* __restrict__ loss, float* __restrict__ dLdE) {
  __shared__ double s_warp[kObjThreads / 32];
  __shared__ double s_sum[1], s_tot[1];
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = kObjCluster * kObjThreads;
  const int tid = (int)cl.block_rank() * kObjThreads + threadIdx.x;
  const int ncell = ncol * nrow;
  pdl_trigger();
  pdl_wait();      // E is the previous kernel's output
  float part[1] = {0.0f};
  for (int q0 = tid; q0 < ncell; q0 += kObjUnroll * nthr) {
    float e[kObjUnroll], r[kObjUnroll];
    bool in[kObjUnroll];
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int q = q0 + u * nthr;
      const int row = q / ncol, col = q - row * ncol;
      const int i = col - hx, j = row - hy;
      in[u] = q < ncell && i >= 0 && i < nx && j >= 0 && j < ny;
      e[u] = in[u] ? E[q] : 0.0f;
      r[u] = in[u] ? Eref[(size_t)j * nx + i] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kObjUnroll; ++u) {
      const int q = q0 + u * nthr;
      if (q >= ncell) break;
      const float d = __fsub_rn(e[u], r[u]);
      part[0] = __fmaf_rn(d, d, part[0]);
      dLdE[q] = 2.0f * d;
    }
  }
  cluster_sum<1>(part, s_warp, s_sum, s_tot);
  if (threadIdx.x == 0 && cl.block_rank() == 0) *loss = s_tot[0];
  cl.sync();
}

__global__ void k_reparam_tanh(const float* __restrict__ theta, const float* __restrict__ offset, int64_t n,
                               float z_min, float half_range, float* __restrict__ P) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float base = offset ? offset[k] + z_min : z_min;
  P[k] = fmaf(half_range, tanhf(theta[k]) + 1.0f, base);
}

__global__ void k_reparam_tanh_adjoint(const float* __restrict__ theta, const float* __restrict__ dLdP, int64_t n,
                                       float half_range, float* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float t = tanhf(theta[k]);
  out[k] = dLdP[k] * half_range * fmaf(-t, t, 1.0f);
}

// Adam (Kingma & Ba, Algorithm 1) on theta with the gradient dL/dtheta taken
// from dL/dP through the tanh map, then P rewritten from the new theta. One
// block, so every thread reads the step count before thread 0 advances it.
__global__ void __launch_bounds__(1024) k_adam_tanh(float* __restrict__ theta, float* __restrict__ m,
                                                    float* __restrict__ v, const float* __restrict__ dLdP,
                                                    const float* __restrict__ offset, int64_t n, float lr, float b1,
                                                    float b2, float eps, float z_min, float half_range,
                                                    int32_t* step, float* __restrict__ P) {
  pdl_wait();
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = *step + 1;
  __syncthreads();
  const int t = s_t;
  const float bc1 = 1.0f - powf(b1, (float)t);
  const float bc2 = 1.0f - powf(b2, (float)t);
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    float th = theta[q];
    const float th_t = tanhf(th);
    const float gq = dLdP[q] * half_range * fmaf(-th_t, th_t, 1.0f);
    const float mq = fmaf(b1, m[q], (1.0f - b1) * gq);
    const float vq = fmaf(b2, v[q], (1.0f - b2) * gq * gq);
    m[q] = mq;
    v[q] = vq;
    th -= lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
    theta[q] = th;
    const float base = offset ? offset[q] + z_min : z_min;
    P[q] = fmaf(half_range, tanhf(th) + 1.0f, base);
  }
  if (threadIdx.x == 0) *step = t;
}

// Greville abscissa u*_i = (u_{i+1} + ... + u_{i+p}) / p of the clamped uniform
// knot vector u_k = clamp((k - p) / (n - p + 1), 0, 1).
__device__ double greville(int i, int n, int p) {
  double s = 0.0;
  for (int k = i + 1; k <= i + p; ++k) s += fmin(fmax((double)(k - p) / (double)(n - p + 1), 0.0), 1.0);
  return s / p;
}

// f(P^x_ij, P^y_ij) = c + R - sign(R) sqrt(R^2 - x^2 - y^2) (R = 0: c) at
// P^x_ij = (2u*_i - 1) r_x, P^y_ij = (2v*_j - 1) r_y. The host has checked that
// the sphere covers every control point.
__global__ void k_offset_spherical(int n1, int n2, int p, int q, double rx, double ry, double c, double R,
                                   float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (n1 + 1) * (n2 + 1)) return;
  const int i = k / (n2 + 1), j = k - i * (n2 + 1);
  const double x = (2.0 * greville(i, n1, p) - 1.0) * rx;
  const double y = (2.0 * greville(j, n2, q) - 1.0) * ry;
  double f = c;
  if (R != 0.0) f = c + R - copysign(sqrt(fmax(R * R - x * x - y * y, 0.0)), R);
  out[k] = (float)f;
}

}  // namespace

cudaError_t launch_loss_l2(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y, double* loss,
                           float* dLdE, cudaStream_t st, bool pdl) {
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  return launch_k(k_loss_l2, dim3(kObjCluster), dim3(kObjThreads), 0, st, pdl, E, Eref, nx, ny, (nu_x - 1) / 2,
                  (nu_y - 1) / 2, ncol, nrow, loss, dLdE);
}

cudaError_t launch_loss_frobenius(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y,
                                  double* loss, float* dLdE, cudaStream_t st, bool pdl) {
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  return launch_k(k_loss_frobenius, dim3(kObjCluster), dim3(kObjThreads), 0, st, pdl, E, Eref, nx, ny,
                  (nu_x - 1) / 2, (nu_y - 1) / 2, ncol, nrow, loss, dLdE);
}

cudaError_t launch_reparam_tanh(const float* theta, const float* offset, int64_t n, float z_min, float z_max,
                                float* P, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_reparam_tanh<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, offset, n, z_min, 0.5f * (z_max - z_min), P);
  return cudaGetLastError();
}

cudaError_t launch_reparam_tanh_adjoint(const float* theta, const float* dLdP, int64_t n, float z_min, float z_max,
                                        float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_reparam_tanh_adjoint<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, dLdP, n, 0.5f * (z_max - z_min), out);
  return cudaGetLastError();
}

cudaError_t launch_adam_tanh(float* theta, float* m, float* v, const float* dLdP, const float* offset, int64_t n,
                             float lr, float b1, float b2, float eps, float z_min, float z_max, int32_t* step,
                             float* P, cudaStream_t st, bool pdl) {
  return launch_k(k_adam_tanh, dim3(1), dim3(1024), 0, st, pdl, theta, m, v, dLdP, offset, n, lr, b1, b2, eps, z_min,
                  0.5f * (z_max - z_min), step, P);
}

cudaError_t launch_offset_spherical(int n1, int n2, int p, int q, double rx, double ry, double c, double R,
                                    float* out, cudaStream_t st) {
  const int n = (n1 + 1) * (n2 + 1);
  k_offset_spherical<<<(n + 255) / 256, 256, 0, st>>>(n1, n2, p, q, rx, ry, c, R, out);
  return cudaGetLastError();
}

}  // namespace fr
