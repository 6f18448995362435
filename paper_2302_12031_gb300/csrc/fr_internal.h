// Internal declarations shared by the CUDA translation units of libfreeray.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "freeray.h"

namespace fr {

constexpr int kMaxCtrl = 32;              // control points per direction
constexpr int kMaxSpans = kMaxCtrl - 3;   // knot spans per direction (degree 3)
constexpr int kMaxItems = 64;             // lenses per batched launch

// Device view of one lens problem: lens, source, screen, outputs and schedule.
// Built on the host by the C ABI from the public descriptors.
struct Item {
  // Lens (Sec. 2.1). Spans are the non-empty knot spans of the clamped uniform
  // knot vector: nsu = ncu - p along u, nsv = ncv - q along v (p = q = 3 in
  // every kernel but the general-degree derivative maps).
  const float* ctrl;
  int ncu, ncv, nsu, nsv;
  int p, q;
  float rx, ry, z_in, n_glass;
  float ku, kv;                 // d(span coordinate)/dx = nsu/(2 rx), likewise kv
  float R0;                     // ((n-1)/(n+1))^2
  // Optional freeform entry face (both faces optimised): a second net over the
  // same aperture; two_face = 0: the flat face z = z_in.
  int two_face;
  const float* ctrl_in;
  int ncu_in, ncv_in, nsu_in, nsv_in;
  float ku_in, kv_in;
  int nparam;                   // control heights: ncu ncv (+ ncu_in ncv_in); dL/dP has this many
  // Source (Sec. 2.2.1).
  int kind, jitter, cols, rows;
  uint32_t row_lo, row_hi;      // collimated: the rows of the call's cells [ray_begin, ray_end),
  uint32_t col_lo, col_hi;      // which start at column col_lo of row_lo and end before
                                // column col_hi of row_hi - 1
  float px, py, pz;             // source position (grid centre)
  float omc_max;                // 1 - cos(phi_max)
  int gnx, gny;
  float gx0, gy0, gdx, gdy;     // first grid position offset and spacing
  uint32_t per_src;             // rays per point source of the grid
  uint64_t seed, n_rays;
  uint64_t ray_begin, ray_end;  // rays traced by this call
  const uint32_t* order;        // point sources: the ray at position p is order[p] (NULL: p)
  // Point sources in the hot trace kernels: rays whose intersection needs the
  // march (first_root) are appended here, as offsets from ray_begin, for the
  // deferred pass; defer_n[0] counts them (the deferred pass resets it).
  uint32_t* defer;
  uint32_t* defer_n;
  float omega0;                 // flux / n_rays
  // Screen and filter (Sec. 2.3).
  float z_screen, Rx, Ry;
  int nx, ny, nu, ncol, nrow;
  float inv_wx, inv_wy;         // 1/w
  float Rsx, Rsy;               // R* = R + (nu-1)/2 w
  float gx_off, gy_off;         // R* / w: the screen edge -R* in extended pixel units
  float ax, ay;                 // alpha * log2(e)
  float cut;                    // exp(-alpha (nu/2)^2)
  float inv_area;               // 1/(w_x w_y)
  // Outputs.
  float* E;                     // forward, float mode
  unsigned long long* Efix;     // forward, deterministic mode
  float fixE;                   // fixed-point scale of E (a power of two)
  const float* dLdE;            // adjoint input
  float* dLdP;                  // adjoint, float mode
  unsigned long long* Pfix;     // adjoint, deterministic mode
  const float* gmax;            // adjoint, deterministic: max |dL/dE| (device)
  float fixP_unit;              // adjoint, deterministic: flux / (w_x w_y)
  fr_stats* stats;
  // Newton (Sec. 2.2.1 intersection, point sources).
  int newton_max;
  float newton_tol;
  // Triangle mesh instead of Newton (Sec. 2.2.2, point sources): mesh_nu x
  // mesh_nv rectangles per knot span product, NU = nsu mesh_nu by NV = nsv
  // mesh_nv cells over [0,1]^2; mesh_nu = 0: Newton.
  int mesh_nu, mesh_nv, NU, NV;
  float inv_mnu, inv_mnv;       // 1/mesh_nu, 1/mesh_nv
  // Schedule: the item's rays are split evenly over the lanes of CTAs
  // [cta_begin, cta_end) of the launch (lane_range in fr_device.cuh).
  int max_ctas;                 // CTAs worth launching (every lane gets a minimum run)
  int smem_hist;                // forward: 1 = privatised histogram in shared memory,
                                // 2 = a window of it (rows win_r0..win_r1-1, columns
                                // win_c0..win_c1-1 of the extended grid) in shared memory
  int win_r0, win_r1, win_c0, win_c1;
  int cta_begin, cta_end;
};

template <int CAP>
struct Launch {
  int n_items;
  int warps;                    // warps per CTA
  int early_lens;               // adjoint under programmatic launch: build the lens tables before
                                // waiting for the previous kernel (which must not write the lens)
  Item items[CAP];
};

// Launch with or without programmatic dependent launch: with `pdl` the kernel
// may begin while the previous kernel on the stream is still running; it calls
// pdl_wait() (griddepcontrol.wait) before it reads anything that kernel wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Shared-memory bytes a CTA of the forward / adjoint kernel needs for `it`.
size_t fwd_smem_bytes(const Item& it, bool det);
size_t lens_tables_bytes(const Item& it);   // the lens tables part of it
size_t adj_smem_bytes(const Item& it, bool det);

// Launchers (return the CUDA error of the launch).
// march: a single point-source lens whose intersections march in the kernel
// (no deferred pass; the allocation-free entry point).
template <int CAP>
cudaError_t launch_forward(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st, bool pdl,
                           bool march = false);
// Zeroes up to kMaxZero buffers (sizes in bytes) in one launch.
constexpr int kMaxZero = 80;   // a batch's 64 grids and its dL/dP, with room
struct ZeroList {
  int n;
  void* ptr[kMaxZero];
  uint64_t bytes[kMaxZero];
};
cudaError_t launch_zero_list(const ZeroList& z, cudaStream_t st);
template <int CAP>
cudaError_t launch_adjoint(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st, bool pdl);
cudaError_t launch_debug(const Item& it, fr_ray_record* out, cudaStream_t st);
cudaError_t launch_fix_to_float(const unsigned long long* q, float* out, size_t n, float inv_scale,
                                int accumulate, cudaStream_t st);
cudaError_t launch_absmax(const float* x, size_t n, float* out, cudaStream_t st);
cudaError_t launch_loss_l2(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y, double* loss,
                           float* dLdE, cudaStream_t st, bool pdl);
cudaError_t launch_adam(float* P, float* m, float* v, const float* g, int64_t n, float lr, float b1,
                        float b2, float eps, int32_t* step, cudaStream_t st, bool pdl);
cudaError_t launch_grad_fix_to_float(const Item& it, int accumulate, cudaStream_t st);
cudaError_t launch_loss_frobenius(const float* E, const float* Eref, int nx, int ny, int nu_x, int nu_y,
                                  double* loss, float* dLdE, cudaStream_t st, bool pdl);
cudaError_t launch_reparam_tanh(const float* theta, const float* offset, int64_t n, float z_min, float z_max,
                                float* P, cudaStream_t st);
cudaError_t launch_reparam_tanh_adjoint(const float* theta, const float* dLdP, int64_t n, float z_min,
                                        float z_max, float* out, cudaStream_t st);
cudaError_t launch_adam_tanh(float* theta, float* m, float* v, const float* dLdP, const float* offset, int64_t n,
                             float lr, float b1, float b2, float eps, float z_min, float z_max, int32_t* step,
                             float* P, cudaStream_t st, bool pdl);
cudaError_t launch_offset_spherical(int n1, int n2, int p, int q, double rx, double ry, double c, double R,
                                    float* out, cudaStream_t st);
// Coherent ray order (fr_ray_order): counting sort of the ray ids by source
// and cell (m x m cells per knot span). Scratch: `counts` n_keys words,
// `keys` n_rays words, `partial` ray_order_scratch_words words.
int ray_order_grid(const Item& it);
uint64_t ray_order_keys(const Item& it, int m);
uint64_t ray_order_scratch_words(const Item& it, int m);
cudaError_t launch_ray_order(const Item& it, int m, uint32_t* counts, uint32_t* keys, uint32_t* partial,
                             uint32_t* order, cudaStream_t st);
size_t tan_smem_bytes(const Item& it);
cudaError_t launch_tangent(const Item& it, int warps, int grid, size_t smem, const float* dP, int n_dirs, float* dE,
                           cudaStream_t st);
// Derivative maps of a collimated lens of any degrees 1..5 (p, q of the Item).
size_t tan_general_smem_bytes(const Item& it);
cudaError_t launch_tangent_general(const Item& it, int warps, int grid, const float* dP, int n_dirs, float* dE,
                                   cudaStream_t st);
int tangent_occupancy(int threads, size_t smem, int nu);
cudaError_t configure_tangent(int optin);
cudaError_t configure_forward(int optin);
cudaError_t configure_adjoint(int optin);

// Throughput probes (fr_probe): operations of one launch, and the launch.
double probe_ops(int kind, int blocks, int threads, int iters);
cudaError_t launch_probe(int kind, int blocks, int threads, int iters, float* out, int n_out, cudaStream_t st);

// The deferred pass after a hot point-source trace launch (same Launch, det
// and filter size): traces the items' deferred rays with the march.
template <int CAP>
cudaError_t launch_forward_deferred(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st);
template <int CAP>
cudaError_t launch_adjoint_deferred(const Launch<CAP>& L, int grid, size_t smem, bool det, cudaStream_t st);

// Occupancy of the trace kernels for a block size and dynamic shared memory.
// kinds: 1 collimated, 2 point source, 4 two-face lens, 8 point source marching in
// the kernel (single-lens launches); batches use both of 1 and 2.
int forward_occupancy(int threads, size_t smem, bool det, bool batch, int nu, int kinds);
int adjoint_occupancy(int threads, size_t smem, bool det, bool batch, int nu, int kinds);

}  // namespace fr
