// The paper's objective and parametrisation around the trace:
//  - the normalised Frobenius loss and its gradient (Sec. 2.5, Eq. pipelineLoss),
//    one launch of one thread-block cluster whose CTAs reduce through
//    distributed shared memory in a fixed order (bit-identical run to run, no
//    atomics, no counters, no scratch memory);
//  - control heights from unconstrained variables through tanh onto
//    (z_min, z_max) plus an offset f(P^x, P^y) (Sec. 2.4.2, Eqs. outputcorrection
//    and outputcorrectionwfunc), its adjoint, the spherical offsets of Table
//    magndata at the Greville points (Sec. 2.1), and Adam on the unconstrained
//    variables fused with both maps.
#include <cooperative_groups.h>

#include "fr_internal.h"

namespace cg = cooperative_groups;

namespace fr {
namespace {

constexpr int kObjCluster = 8;      // CTAs of the loss cluster (portable cluster size)
constexpr int kObjThreads = 512;

// Sums NV doubles over the cluster: a fixed xor tree in each warp, then over
// the warps of the CTA, then over the CTAs in rank order through distributed
// shared memory. Every thread of the cluster returns the same totals in v.
// s_cta is this call's own slot (it is read by the other CTAs after the
// cluster barrier, so a later call must use another slot, and the kernel must
// pass one more cluster barrier before it exits).
template <int NV>
__device__ __forceinline__ void cluster_sum(double (&v)[NV], double* s_warp, double* s_cta) {
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_warp[warp * NV + k] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < (int)(blockDim.x >> 5) ? s_warp[lane * NV + k] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) s_cta[k] = x;
    }
  }
  cl.sync();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = 0.0;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) t += *cl.map_shared_rank(s_cta + k, r);
    v[k] = t;
  }
}

// With I^ = E/S, I^_ref = E_ref/S_ref over the interior and D = I^ - I^_ref:
// L = ||D||_F / sqrt(nx ny), and dL/dE = (c D - c sum(D I^)) / S on the interior
// with c = 1/(sqrt(nx ny) ||D||_F), 0 on ghost pixels. ||D|| = 0 gives a zero
// gradient; S <= 0 or S_ref <= 0 gives L = NaN and a zero gradient.
__global__ void __cluster_dims__(kObjCluster, 1, 1) __launch_bounds__(kObjThreads)
    k_loss_frobenius(const float* __restrict__ E, const float* __restrict__ Eref, int nx, int ny, int hx, int hy,
                     int ncol, int nrow, double* __restrict__ loss, float* __restrict__ dLdE) {
  __shared__ double s_warp[(kObjThreads / 32) * 2];
  __shared__ double s_sums[2], s_dots[2];
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = kObjCluster * kObjThreads;
  const int tid = (int)cl.block_rank() * kObjThreads + threadIdx.x;
  const int n = nx * ny;

  double s[2] = {0.0, 0.0};
  for (int k = tid; k < n; k += nthr) {
    const int j = k / nx, i = k - j * nx;
    s[0] += (double)E[(size_t)(j + hy) * ncol + (i + hx)];
    s[1] += (double)Eref[k];
  }
  cluster_sum<2>(s, s_warp, s_sums);
  const bool ok = s[0] > 0.0 && s[1] > 0.0;
  // I^ and I^_ref by correctly rounded division (not by a reciprocal): images
  // equal up to a power-of-two scale then give D = 0 exactly, where the norm's
  // gradient would otherwise point along rounding noise.
  const double S = ok ? s[0] : 1.0, Sr = ok ? s[1] : 1.0;

  double d2[2] = {0.0, 0.0};          // sum D^2, sum D I^
  for (int k = tid; k < n; k += nthr) {
    const int j = k / nx, i = k - j * nx;
    const double I = (double)E[(size_t)(j + hy) * ncol + (i + hx)] / S;
    const double D = I - (double)Eref[k] / Sr;
    d2[0] = fma(D, D, d2[0]);
    d2[1] = fma(D, I, d2[1]);
  }
  cluster_sum<2>(d2, s_warp, s_dots);
  const double root_n = sqrt((double)nx * (double)ny);
  const double norm = sqrt(d2[0]);
  const double c = (ok && norm > 0.0) ? 1.0 / (root_n * norm) : 0.0;
  const double gdot = c * d2[1];

  for (int q = tid; q < ncol * nrow; q += nthr) {
    const int r = q / ncol, col = q - r * ncol;
    const int i = col - hx, j = r - hy;
    float g = 0.0f;
    if (c != 0.0 && i >= 0 && i < nx && j >= 0 && j < ny) {
      const double I = (double)E[q] / S;
      const double D = I - (double)Eref[(size_t)j * nx + i] / Sr;
      g = (float)((c * D - gdot) / S);
    }
    dLdE[q] = g;
  }
  if (tid == 0) *loss = ok ? norm / root_n : __longlong_as_double(0x7ff8000000000000LL);
  cl.sync();       // no CTA leaves while another may still read its shared memory
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

cudaError_t launch_loss_frobenius(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y,
                                  double* loss, float* dLdE, cudaStream_t st) {
  const int ncol = nx + nu_x - 1, nrow = ny + nu_y - 1;
  k_loss_frobenius<<<kObjCluster, kObjThreads, 0, st>>>(E, Eref, nx, ny, (nu_x - 1) / 2, (nu_y - 1) / 2, ncol,
                                                        nrow, loss, dLdE);
  return cudaGetLastError();
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
                             float* P, cudaStream_t st) {
  k_adam_tanh<<<1, 1024, 0, st>>>(theta, m, v, dLdP, offset, n, lr, b1, b2, eps, z_min, 0.5f * (z_max - z_min),
                                  step, P);
  return cudaGetLastError();
}

cudaError_t launch_offset_spherical(int n1, int n2, int p, int q, double rx, double ry, double c, double R,
                                    float* out, cudaStream_t st) {
  const int n = (n1 + 1) * (n2 + 1);
  k_offset_spherical<<<(n + 255) / 256, 256, 0, st>>>(n1, n2, p, q, rx, ry, c, R, out);
  return cudaGetLastError();
}

}  // namespace fr
