/*
 * freeray — C ABI of the GB300 (sm_103a) differentiable freeform-lens tracer.
 *
 * Implements the hot path of de Koning, Heemels, Adam and Moeller, "Gradient
 * descent-based freeform optics design using algorithmic differentiable
 * non-sequential ray tracing" (2023): rays from a collimated beam, a point
 * source or a grid of point sources are traced through a lens made of a flat
 * entry face and a bicubic B-spline freeform exit face (Sec. 2.1) onto a screen,
 * deposited with the smooth Gaussian reconstruction filter (Sec. 2.3), and the
 * gradient of an irradiance loss is carried back to the control heights P^z
 * (Sec. 2.5).
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" are CUDA device (or managed) memory owned
 *    by the caller; the library never frees them. Pointers documented as
 *    "host" are read during the call only.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    enqueued on it asynchronously; nothing in this library synchronises the
 *    host with the device, except fr_stream_wait (explicitly).
 *  - Every call returns an fr_status. On failure nothing has been enqueued
 *    (argument errors) or the CUDA error is reported (launch errors); a message
 *    is kept in the handle (fr_last_error). No exception crosses the ABI and no
 *    kernel traps: per-ray anomalies are counted in fr_stats.
 *  - Calls taking an fr_handle allocate device scratch memory in the handle the
 *    first time a larger problem is seen (the fixed-point accumulators, and for
 *    a point source intersected by Newton a list of 4 bytes per traced ray: the
 *    rays whose smallest root needs the certified march are traced again by a
 *    second kernel right after the first). That allocation is refused with
 *    FR_ERR_WORKSPACE while `stream` is being captured into a CUDA graph, so a
 *    call of the same size must run once before capture. A point-source call
 *    traces at most 2^32 - 1 rays.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Only clamped uniform knot vectors and degrees p = q = 3 are supported,
 *    except that a collimated single-face lens may have degrees p, q from 1
 *    to 5 in fr_trace_forward, fr_trace_adjoint and fr_trace_tangent (one
 *    lens per call; general-degree kernels evaluate each ray's basis
 *    functions by the Cox-de Boor recursion);
 *    control nets from 4x4 to 32x32; filter sizes nu_x = nu_y odd, 1 to 11.
 *    Sizes 7 to 11 run in the wide-filter trace kernels: one single-face lens
 *    per call (FR_ERR_UNSUPPORTED for a batch or a freeform entry face), not
 *    in fr_trace_forward_static.
 *
 * Layouts:
 *  - Control heights: float32, (n1+1) x (n2+1), row-major with the u index i
 *    slow: ctrl_z[i*(n2+1) + j] = P^z_{i,j}; u runs along x, v along y.
 *  - Irradiance and dL/dE: float32 on the extended grid with ghost pixels
 *    (Sec. 2.3), (ny+nu_y-1) rows x (nx+nu_x-1) columns, row-major, row = y:
 *    E[r*(nx+nu_x-1) + c]. Interior pixel (i, j) is column i+(nu_x-1)/2,
 *    row j+(nu_y-1)/2. Units: flux per area, E = sum_k w_k F(x_k) / (w_x w_y).
 *  - Target images for the loss: float32 on the interior ny x nx grid.
 */
#ifndef FREERAY_H
#define FREERAY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Version 2: fr_options.ray_order and window_cells, fr_batch_item.ray_order.
 * Version 3: fr_options.batch_waves (in place of a reserved word). */
#define FR_ABI_VERSION 3

typedef enum fr_status {
  FR_OK = 0,
  FR_ERR_INVALID_ARG = 1,  /* a descriptor or size is out of range */
  FR_ERR_UNSUPPORTED = 2,  /* valid, but outside what this build implements */
  FR_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
  FR_ERR_WORKSPACE = 4,    /* scratch memory needed while a stream is capturing */
  FR_ERR_TIMEOUT = 5       /* fr_stream_wait ran out of time */
} fr_status;

/* Source kinds (Sec. 2.2.1). */
enum { FR_SOURCE_COLLIMATED = 0, FR_SOURCE_POINT = 1 };

/* What happened to a ray; index into fr_stats.rays and fr_ray_record.status. */
enum {
  FR_RAY_ON_SCREEN = 0,     /* deposited */
  FR_RAY_APERTURE_MISS = 1, /* point source: missed the entry face */
  FR_RAY_OUT_OF_DOMAIN = 2, /* point source: left the side of the lens before the freeform */
  FR_RAY_TIR = 3,           /* total internal reflection at the freeform (culled, Sec. 2.2) */
  FR_RAY_OFF_SCREEN = 4,    /* missed the open interior screen |X|<R_x, |Y|<R_y */
  FR_RAY_INVALID = 5,       /* freeform below the entry face where the ray enters */
  FR_RAY_NEWTON_FAIL = 6,   /* point source: the intersection did not converge in its evaluations */
  FR_RAY_NCAUSES = 8
};

/* Lens (Sec. 2.1): flat entry face z = z_in on [-rx,rx]x[-ry,ry] and the
 * freeform z = Z(X^-1(x), Y^-1(y)), a B-spline of degrees (p, q) over clamped
 * uniform knots whose X and Y are linear through the Greville construction. */
typedef struct fr_lens_desc {
  int32_t n1, n2;        /* control net (n1+1) x (n2+1); 3 <= n1, n2 <= 31 */
  int32_t p, q;          /* degrees; must be 3 */
  const float* ctrl_z;   /* device, (n1+1)*(n2+1) control heights P^z */
  float rx, ry;          /* half-widths of the lens */
  float z_in;            /* entry face; P^z > z_in keeps the lens valid (Sec. 2.1.2) */
  float n_glass;         /* refractive index of the lens; air outside */
  /* Optional freeform entry face (both faces optimised, as the paper's
   * conclusion proposes): NULL = the flat face z = z_in; else device,
   * (entry_n1+1)*(entry_n2+1) heights of a second bicubic net over the same
   * aperture (same layout as ctrl_z). The lens is valid where the entry face
   * lies below the exit face. With an entry face, dL/dP outputs hold the exit
   * net's gradient followed by the entry net's. Single-lens calls only (not
   * in batches, not with the triangle mesh, not for fr_trace_tangent). */
  const float* entry_ctrl_z;
  int32_t entry_n1, entry_n2;
} fr_lens_desc;

/* Source (Sec. 2.2.1). Rays are numbered 0..n_rays-1; the initial weight of
 * every ray is flux / n_rays. */
typedef struct fr_source_desc {
  int32_t kind;          /* FR_SOURCE_COLLIMATED or FR_SOURCE_POINT */
  int32_t jitter;        /* collimated: 0 = cell centres, 1 = Philox jitter in each cell */
  int32_t cols, rows;    /* collimated: square grid over (u,v) in [0,1]^2, n_rays = cols*rows,
                            ray id = row*cols + col */
  float pos[3];          /* point: source position (centre of the grid of sources) */
  float half_angle;      /* point: cone half-angle phi_max in radians, (0, pi/2) */
  int32_t grid_nx, grid_ny; /* point: grid of point sources (1,1 for one source);
                               n_rays must be a multiple of grid_nx*grid_ny */
  float grid_w, grid_h;  /* point: extent of the grid; centres equispaced including the ends */
  float flux;            /* total flux of the source */
} fr_source_desc;

/* Screen and reconstruction filter (Sec. 2.3). */
typedef struct fr_target_desc {
  float z_screen;        /* screen plane, above the lens */
  float Rx, Ry;          /* screen half-widths; pixel size w = 2R/n */
  int32_t nx, ny;        /* interior pixels, 1..4096 */
  int32_t nu_x, nu_y;    /* filter sizes (odd, equal, 1..11) */
  float alpha;           /* Gaussian coefficient in pixel units: exp(-alpha ((x-c)/w)^2) */
} fr_target_desc;

/* Options. Zero-initialised options mean the defaults. */
typedef struct fr_options {
  int32_t deterministic;    /* 1: accumulate in int64 fixed point; results are bit-identical
                               from run to run and independent of the launch schedule */
  int32_t accumulate;       /* 1: add into E_out / dLdP_out instead of overwriting them */
  int32_t newton_max_iter;  /* 0 -> 8: Newton iterations towards the smallest root
                               (Sec. 2.2.1; where the bounds cannot certify Newton's root the
                               certified march takes at most 32 evaluations more) */
  float newton_tol;         /* 0 -> 1e-6, absolute, on the ray parameter */
  int32_t warps_per_cta;    /* 0 -> tuned; 1..32 */
  int32_t rays_per_lane;    /* 0 -> tuned; 1..64 */
  int32_t ctas_per_sm;      /* 0 -> tuned; 1..8 */
  int32_t hist_mode;        /* 0 auto, 1 global atomics, 2 shared-memory privatised,
                               3 shared-memory window (point sources, float mode): the central
                               part of the extended grid that fits in shared memory is
                               privatised, deposits outside it go to global memory; auto picks
                               it for a point source whose extended grid does not fit */
  void* event_begin;        /* optional cudaEvent_t, recorded on the stream right before the
                               trace kernel (not the prep or conversion kernels) */
  void* event_end;          /* optional cudaEvent_t, recorded right after the trace kernel */
  int32_t mesh_nu;          /* point sources: 0 -> Newton on the B-spline (Sec. 2.2.1); n > 0 ->
                               the triangle mesh of Sec. 2.2.2 with mesh_nu x mesh_nv rectangles
                               (two triangles each) per knot span product; 1..64 */
  int32_t mesh_nv;          /* 0 with mesh_nu = 0, else 1..64 */
  const uint32_t* ray_order; /* point sources, optional (device): the n_rays + 1 words written
                               by fr_ray_order, in whose order the forward, adjoint and
                               derivative-map traces take the rays; the sums are over the
                               same rays. Only for calls over all rays of one lens
                               (FR_ERR_INVALID_ARG else); NULL: id order */
  int32_t window_cells;     /* hist_mode 3: at most this many cells in the window; 0 -> as
                               many as shared memory holds */
  int32_t batch_waves;      /* batched calls: the launch holds this many waves of CTAs (items
                               get CTAs in proportion to their cost, so unequal items balance
                               over the waves); 0 -> 8, at most 64 */
  int32_t reserved[2];
} fr_options;

/* Per-cause ray counts (device, uint64). Kernels add to it; zero it first. */
typedef struct fr_stats {
  uint64_t rays[FR_RAY_NCAUSES];
} fr_stats;

/* One traced ray, for debugging and parity checks (fr_trace_debug). */
typedef struct fr_ray_record {
  int32_t status;        /* FR_RAY_* */
  int32_t span_i, span_j;/* knot span index of the freeform hit (u_i0 <= u < u_i0+1) */
  int32_t newton_iters;  /* point source: Newton iterations used */
  float u, v;            /* freeform hit, parameter space */
  float x, y, z;         /* freeform hit */
  float dx, dy, dz;      /* direction inside the glass */
  float tx, ty, tz;      /* direction after the freeform */
  float X, Y;            /* screen hit */
  float w;               /* final weight */
  float t;               /* point source: ray parameter of the hit inside the glass */
} fr_ray_record;

/* One lens of a batched call: its own descriptors, rays and buffers. */
typedef struct fr_batch_item {
  fr_lens_desc lens;
  fr_source_desc source;
  fr_target_desc target;
  uint64_t n_rays;
  uint64_t seed;
  float* E;              /* device: forward output, extended grid */
  const float* dLdE;     /* device: adjoint input, extended grid */
  float* dLdP;           /* device: adjoint output, (n1+1)*(n2+1) */
  fr_stats* stats;       /* device or NULL */
  const uint32_t* ray_order; /* point source, optional (device): this item's fr_ray_order
                               output (as fr_options.ray_order for one lens); NULL: id order */
} fr_batch_item;

typedef struct fr_handle fr_handle;

/* Create / destroy a handle bound to the current CUDA device. */
fr_status fr_create(fr_handle** out);
fr_status fr_destroy(fr_handle* h);

/* Message of the last failure on this handle ("" if none). Valid until the next
 * call. With h == NULL: the last failure on this host thread of a call made
 * without a handle (fr_create, fr_trace_forward_static; the latter clears it
 * when it starts, so after a successful call it is ""). */
const char* fr_last_error(const fr_handle* h);

/* ABI version (FR_ABI_VERSION) of the loaded library. */
int32_t fr_abi_version(void);

/* Forward trace (Secs. 2.2-2.3): rays [ray_begin, ray_begin+ray_count) of a
 * source of n_rays rays through the lens onto the screen. Writes (or adds, with
 * options->accumulate) the irradiance on the extended grid to E_out (device),
 * and adds per-cause ray counts to stats_out (device, may be NULL).
 * ray_count = UINT64_MAX means "to the end". `seed` keys the Philox stream of
 * the point source and of collimated jitter. options may be NULL. */
fr_status fr_trace_forward(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                           uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                           float* E_out, fr_stats* stats_out, void* stream);

/* Adjoint (reverse mode of the forward trace, Sec. 2.5): given dL/dE on the
 * extended grid (device), writes (or adds) dL/dP^z to dLdP_out (device,
 * (n1+1)*(n2+1), followed by (entry_n1+1)*(entry_n2+1) for a freeform entry
 * face). Each ray's path is recomputed from its id and seed, not read
 * back; the arguments must equal those of the forward call. */
fr_status fr_trace_adjoint(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                           uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                           const float* dLdE, float* dLdP_out, fr_stats* stats_out, void* stream);

/* Forward mode (the irradiance derivatives of Sec. 3.1): for n_dirs (1..32)
 * directions dP_k in control-height space, dP device n_dirs x (n1+1)*(n2+1)
 * (direction k at dP + k*(n1+1)*(n2+1), control-height layout), writes (or
 * adds) the directional derivatives dE_k = sum_ij (dE/dP^z_ij) dP_k,ij of the
 * irradiance over rays [ray_begin, ray_begin+ray_count) to dE_out (device,
 * n_dirs extended grids, grid k at dE_out + k*(nx+nu_x-1)*(ny+nu_y-1)). The
 * derivative map of one control point is dP = its unit vector. Same lens,
 * source, screen and rays as fr_trace_forward; deposits use float atomics
 * (not bit-reproducible; options.deterministic is ignored). For a collimated
 * source the lens may also have degrees p, q from 1 to 5 (at least p + 1 and
 * q + 1 control points; the Sec. 3.1 figure shows (5,3) beside (3,3)): a
 * second kernel evaluates each ray's basis functions by the Cox-de Boor
 * recursion; other degrees with a point source: FR_ERR_UNSUPPORTED. */
fr_status fr_trace_tangent(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                           uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                           const float* dP, int32_t n_dirs, float* dE_out, fr_stats* stats_out, void* stream);

/* Per-ray records of rays [ray_begin, ray_begin+ray_count) (device array of
 * ray_count records). Same path as fr_trace_forward. */
fr_status fr_trace_debug(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                         const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                         uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                         fr_ray_record* out, void* stream);

/* Squared L2 loss over the interior pixels, L = sum (E - E_ref)^2, into
 * *loss_out (a double in device memory, or in pinned host memory, which the
 * kernel writes through unified addressing: no copy needed to read it on the
 * host after the stream completes), and dL/dE = 2 (E - E_ref) on the interior
 * and 0 on ghost pixels into dLdE_out (device, extended grid). E is on the extended
 * grid, E_ref on the interior ny x nx grid. The sum is reduced in a fixed order
 * (bit-identical run to run). */
fr_status fr_loss_l2(fr_handle* h, const float* E, const float* E_ref, int32_t nx, int32_t ny,
                     int32_t nu_x, int32_t nu_y, double* loss_out, float* dLdE_out, void* stream);

/* Adam (Kingma & Ba, Algorithm 1) on n parameters in place (device P, m, v;
 * gradient g). *step (device int32) is the number of steps taken so far: the
 * update uses step+1 for the bias corrections and stores step+1, so a captured
 * graph can be replayed. */
fr_status fr_adam_step(fr_handle* h, float* P, float* m, float* v, const float* g, int64_t n,
                       float lr, float beta1, float beta2, float eps, int32_t* step, void* stream);

/* The paper's loss (Sec. 2.5, Eq. pipelineLoss): with the interior images
 * normalised to unit sum, I^ = E / sum(E) and I^_ref = E_ref / sum(E_ref),
 * L = ||I^ - I^_ref||_F / sqrt(nx ny) into *loss_out (device double or
 * pinned host memory, as for fr_loss_l2), and dL/dE through both
 * normalisations into dLdE_out (device, extended grid; 0 on ghost
 * pixels). E is on the extended grid, E_ref on the interior ny x nx grid.
 * Where ||I^ - I^_ref|| = 0 the gradient is 0. Where sum(E) <= 0 or
 * sum(E_ref) <= 0 the normalisation is undefined: *loss_out is NaN and the
 * gradient 0 (reported on the device, not by the return code). Sums are
 * reduced in a fixed order (bit-identical run to run). Needs no scratch. */
fr_status fr_loss_frobenius(fr_handle* h, const float* E, const float* E_ref, int32_t nx, int32_t ny,
                            int32_t nu_x, int32_t nu_y, double* loss_out, float* dLdE_out, void* stream);

/* Control heights from unconstrained variables (Sec. 2.4.2, Eqs.
 * outputcorrection and outputcorrectionwfunc):
 *   P[k] = offset[k] + z_min + (tanh(theta[k]) + 1) (z_max - z_min) / 2,
 * theta, offset and P_out device arrays of n floats; offset may be NULL (0).
 * Requires z_min < z_max, both finite. P_out may alias offset. */
fr_status fr_reparam_tanh(fr_handle* h, const float* theta, const float* offset, int64_t n, float z_min,
                          float z_max, float* P_out, void* stream);

/* Its adjoint: dLdtheta_out[k] = dLdP[k] (z_max - z_min)/2 (1 - tanh^2(theta[k]))
 * (device arrays of n floats). */
fr_status fr_reparam_tanh_adjoint(fr_handle* h, const float* theta, const float* dLdP, int64_t n, float z_min,
                                  float z_max, float* dLdtheta_out, void* stream);

/* Offsets f(P^x_ij, P^y_ij) of eq. outputcorrectionwfunc at the control points
 * of `lens` (its n1, n2, p, q, rx, ry; ctrl_z is not read), with P^x_ij =
 * (2u*_i - 1) r_x and P^y_ij = (2v*_j - 1) r_y at the Greville abscissae u*, v*
 * (Sec. 2.1). f is the spherical cap of Table magndata,
 *   f(x, y) = c + R - sign(R) sqrt(R^2 - x^2 - y^2),
 * a sphere of radius |R| through (0, 0, c); R = 0 gives the constant c.
 * offset_out: device, (n1+1)*(n2+1) floats in the control-height layout.
 * FR_ERR_INVALID_ARG if the sphere does not reach every control point
 * (R^2 < r_x^2 + r_y^2). */
fr_status fr_offset_spherical(fr_handle* h, const fr_lens_desc* lens, float c, float R, float* offset_out,
                              void* stream);

/* Adam (as fr_adam_step) on the unconstrained variables theta, taking
 * dL/dtheta from dL/dP (device, n) through the tanh map of fr_reparam_tanh, and
 * then writing P_out from the updated theta, in one kernel. theta, m, v are
 * updated in place; offset may be NULL. */
fr_status fr_adam_step_tanh(fr_handle* h, float* theta, float* m, float* v, const float* dLdP, const float* offset,
                            int64_t n, float lr, float beta1, float beta2, float eps, float z_min, float z_max,
                            int32_t* step, float* P_out, void* stream);

/* Batched forward / adjoint: every item (its own lens, source, screen, rays and
 * buffers) in one launch of the trace kernel. Same semantics per item as
 * fr_trace_forward / fr_trace_adjoint over all rays of the item. n_items <= 64;
 * the items must share the filter size (FR_ERR_UNSUPPORTED otherwise). */
fr_status fr_trace_batch_forward(fr_handle* h, const fr_batch_item* items, int32_t n_items,
                                 const fr_options* options, void* stream);
fr_status fr_trace_batch_adjoint(fr_handle* h, const fr_batch_item* items, int32_t n_items,
                                 const fr_options* options, void* stream);

/* Programmatic dependent launch for this handle's later calls: when enabled,
 * the loss kernels, the adjoint trace kernel (float mode) and the Adam kernels
 * are launched so that they may begin while the previous kernel on the stream
 * is still running (their blocks start, then wait on the device for that
 * kernel to complete before reading anything). This hides launch latency
 * between the kernels of an optimisation step, most of all inside a CUDA
 * graph. The waits are in the kernels: a call that follows a kernel of another
 * library behaves the same.
 *   mode 0: off (default); 1: on; 2: on, and the adjoint also builds its lens
 *   tables (reads ctrl_z) before it waits: only when the kernel right before
 *   the adjoint does not write the control heights (true for forward -> loss
 *   -> adjoint -> Adam steps); in mode 2 a float-mode forward with
 *   accumulate = 1 also starts early: it builds its tables and, with a
 *   shared-memory histogram, traces all its rays before it waits, so the
 *   kernel right before it must write neither the control heights nor read or
 *   write E except to clear it (true after fr_zero_list of E and dL/dP in a
 *   step). FR_ERR_INVALID_ARG for other modes. */
fr_status fr_set_programmatic_launch(fr_handle* h, int32_t mode);

/* Zeroes `bytes` bytes of device memory at `ptr` on `stream` (a memset node
 * when captured): for clearing outputs that later calls accumulate into. */
fr_status fr_zero(fr_handle* h, void* ptr, uint64_t bytes, void* stream);

/* Zeroes n (0..80) device buffers, ptrs[k] of bytes[k] bytes (host arrays), in
 * one kernel on `stream`: for clearing a step's outputs (E, dL/dP) before its
 * traces accumulate into them. The kernel lets the next kernel begin launching
 * at once (programmatic launch); a forward in mode 2 waits for it before its
 * first write. */
fr_status fr_zero_list(fr_handle* h, void* const* ptrs, const uint64_t* bytes, int32_t n, void* stream);

/* A coherent order of the rays of a point source or grid of point sources
 * (the rays of Sec. 2.2.1). order_out (device, n_rays + 1 uint32) receives a
 * permutation of the ray ids 0..n_rays-1 followed by a count H: positions
 * 0..H-1 hold the rays that meet the aperture, grouped by source and, within a
 * source, sorted by cell: the ray refracted at the entry plane z = z_in is
 * followed to the plane z = z_in + h (h the mean control height of the exit
 * net minus z_in, at the call; 0 if negative), where each knot span of the
 * exit net (in x, y) is cut into m x m cells, the spans taken in row order and
 * the cells of a span in Z order (m the largest power of two up to 128 that
 * leaves 16 or more of a source's rays per cell, else 1), and after the
 * cells the rays whose point there lies outside the aperture; positions
 * H..n_rays-1 hold rays that miss the aperture (the test has a 1e-5 relative
 * margin toward "meets", so a ray placed among the misses misses in the trace
 * too). With this order (fr_options.ray_order) the
 * traces split only the H rays over their lanes and count the others as
 * aperture misses: no warp idles on misses, rays next to each other meet the
 * same knot spans and land on the same pixels, and their Newton iterations
 * agree. The order is a function of the source, the aperture (rx, ry, z_in),
 * the net's size, the mean control height, n_rays and seed; every permutation
 * gives the same sums, so one order serves every optimisation step (as the
 * heights move it only grows less coherent). Within a cell the order is the order of arrival (it may
 * differ from call to call); deterministic-mode results do not depend on it.
 * With a freeform entry face (entry_ctrl_z) the same key orders the rays but
 * H = n_rays: the entry face decides the aperture in the trace. Needs n_rays
 * < 2^32; uses the handle's workspace (4 bytes per cell and per ray);
 * asynchronous on `stream`. FR_ERR_UNSUPPORTED for collimated sources. */
fr_status fr_ray_order(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source, uint64_t n_rays,
                       uint64_t seed, uint32_t* order_out, void* stream);

/* Wait for `stream` on the host by polling, at most timeout_ms milliseconds.
 * Returns FR_ERR_TIMEOUT if the work has not finished by then. */
fr_status fr_stream_wait(fr_handle* h, void* stream, int32_t timeout_ms);

/* Throughput probe: a measurement aid for the roofline of the trace kernels,
 * not an operation of the paper. Launches `blocks` x `threads` threads
 * (threads a multiple of 32, at most 1024) of one probe kernel on `stream`,
 * each doing `iters` rounds of independent operations of one kind:
 *   0 FP32 FMA, 1 packed FP32 FMA pairs (fma.rn.f32x2): *ops_out = flops (FMA = 2);
 *   2 ex2.approx, 3 rsqrt.approx, 4 float -> int -> float conversions:
 *     *ops_out = thread operations on the XU pipe;
 *   5 u32, 6 f32 shared-memory atomic adds at random addresses of a 64 KB
 *     table: *ops_out = atomic thread operations;
 *   7 16-byte float4 reductions (red.global.add.v4.f32) at random addresses
 *     of buf: *ops_out = reductions.
 * buf (device, n_buf >= 4 floats, caller-owned; for kind 7 n_buf is 4 times
 * a power of two) receives per-thread results (kinds 0-6) or the reductions.
 * *ops_out (host) is written before the launch; the caller times the launch
 * (CUDA events on `stream`) and divides. */
fr_status fr_probe(fr_handle* h, int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float* buf,
                   int32_t n_buf, double* ops_out, void* stream);

/* Forward trace that allocates nothing (the paper has no counterpart; this is
 * an interface for callers that cannot allocate device memory: code running in
 * a host process whose device memory is owned by another allocator or budget,
 * real-time loops that cannot afford cudaMalloc's implicit synchronisation,
 * and plug-ins that may only use the buffers they are handed).
 * Same arguments and results as fr_trace_forward, without a handle: the
 * caller passes the lens, source, screen and the output E_out (and stats_out);
 * the scratch memory this trace needs (the int64 accumulator of the
 * fixed-point kernel) lives in one static device array of 1 MiB that every GPU
 * loading the library holds until the process exits. No cudaMalloc, cudaFree
 * or other allocating call is made. The kernel, its schedule and so its
 * results are those of fr_trace_forward for every lens it takes (flat or
 * freeform entry face, any source), with one exception: a float-mode problem
 * whose grid fits neither in shared memory nor in the array as fixed point
 * (more than 122,000 extended cells, not a point source) deposits with float
 * atomics in global memory, the same sums in another rounding order.
 *  - Limits: control nets up to 32x32 (as fr_trace_forward); in deterministic
 *    mode the extended grid (nx+nu_x-1)*(ny+nu_y-1) may have at most 122,000
 *    cells. Larger problems are rejected with FR_ERR_WORKSPACE and a message.
 *  - The first call on a device, with that device current, sets it up: it looks
 *    up the device address of the static array (cudaGetSymbolAddress) and sets
 *    the kernels' shared-memory limit. Make that first call before any stream
 *    capture.
 *  - All calls share the one array and it keeps the last call's contents; the
 *    call clears what must start at zero. Calls whose work overlaps on the GPU
 *    (on different streams, or from different host threads) race on it:
 *    serialise them.
 *  - Errors are reported by the return code and fr_last_error(NULL). */
fr_status fr_trace_forward_static(const fr_lens_desc* lens, const fr_source_desc* source,
                                  const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                                  uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                                  float* E_out, fr_stats* stats_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FREERAY_H */
