// The C ABI of include/freeray.h: argument checks, the device view of each
// problem (fr::Item), the handle's scratch memory, the schedule, and the launch
// sequence of every entry point. All arithmetic of the path runs in the kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fr_internal.h"

struct fr_handle {
  int device = 0;
  int sm_count = 0;
  int smem_optin = 0;           // max dynamic + static shared memory per block
  unsigned char* ws = nullptr;   // scratch memory owned by the handle
  size_t ws_bytes = 0;
  std::string err;
  // CTAs per SM of a trace kernel, by (adjoint, det, batch, nu, kinds, threads, smem).
  std::map<std::tuple<int, int, int, int, int, int, size_t>, int> occupancy;
  bool pdl = false;             // programmatic dependent launch for loss, adjoint and Adam
  bool pdl_early = false;       // ... with the adjoint reading the lens before its wait
};

namespace {

using fr::Item;

// An NVTX range around each entry point (visible to Nsight tools; without a
// tool attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

constexpr size_t kAlign = 256;
// Reserved at the start of the workspace: the counters of the deferred lists
// (two words per item of a launch: the count and the deferred pass's CTA
// ticket), zeroed when the workspace is allocated and left at zero by every
// deferred pass.
constexpr size_t kHeaderBytes = 4 * kAlign;
static_assert(kHeaderBytes >= 2 * sizeof(uint32_t) * fr::kMaxItems, "deferred-list counters");

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

thread_local std::string g_err;   // failures without a handle (fr_create)

fr_status set_error(fr_handle* h, fr_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_err = buf;
  return s;
}

fr_status cuda_error(fr_handle* h, cudaError_t e, const char* what) {
  return set_error(h, FR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FR_CUDA(h, call, what)                         \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_error(h, e_, what); \
  } while (0)

bool finite(float x) { return std::isfinite(x); }

fr_options defaults(const fr_options* o) {
  fr_options d;
  std::memset(&d, 0, sizeof d);
  if (o) d = *o;
  if (d.newton_max_iter <= 0) d.newton_max_iter = 8;
  if (!(d.newton_tol > 0.0f)) d.newton_tol = 1e-6f;
  return d;
}

// Per-item offsets into the workspace: the int64 accumulators of deterministic
// mode, max |dL/dE| and the deferred list of a point source (4 bytes a ray of
// the call: the worst case, every ray deferred).
struct ItemWs {
  size_t efix, pfix, gmax, defer, end;
};

// Whether the hot trace kernels may defer an item's rays (single-face point
// sources intersected by Newton).
// The wide-filter kernels (nu > 5) march in the kernel: no deferred list.
bool may_defer(const Item& it) {
  return it.kind == FR_SOURCE_POINT && !it.two_face && it.mesh_nu == 0 && it.nu <= 5;
}

ItemWs plan(const Item& it, size_t at, bool det_fwd, bool det_adj) {
  ItemWs w;
  w.efix = at;
  if (det_fwd) at = align_up(at + (size_t)it.ncol * it.nrow * sizeof(unsigned long long));
  w.pfix = at;
  if (det_adj) at = align_up(at + (size_t)it.nparam * sizeof(unsigned long long));
  w.gmax = at;
  at = align_up(at + sizeof(float));
  w.defer = at;
  if (may_defer(it)) at = align_up(at + (it.ray_end - it.ray_begin) * sizeof(uint32_t));
  w.end = at;
  return w;
}

fr_status ensure_workspace(fr_handle* h, size_t bytes, cudaStream_t st) {
  if (bytes <= h->ws_bytes) return FR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FR_CUDA(h, cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone)
    return set_error(h, FR_ERR_WORKSPACE,
                     "scratch memory must grow to %zu bytes while the stream is capturing; run the same call "
                     "once before capture", bytes);
  if (h->ws) {
    FR_CUDA(h, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    FR_CUDA(h, cudaFree(h->ws), "cudaFree");
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t want = std::max<size_t>(bytes, 1 << 20);
  FR_CUDA(h, cudaMalloc(&h->ws, want), "cudaMalloc(workspace)");
  FR_CUDA(h, cudaMemset(h->ws, 0, kHeaderBytes), "cudaMemset(workspace header)");
  h->ws_bytes = want;
  return FR_OK;
}

// Checks the public descriptors and fills the device view.
// any_degree: degrees 1..5 (the general-degree derivative maps); else p = q = 3.
fr_status make_item(fr_handle* h, const fr_lens_desc* L, const fr_source_desc* S, const fr_target_desc* T,
                    uint64_t n_rays, uint64_t seed, uint64_t begin, uint64_t count, const fr_options& o,
                    Item* it, bool any_degree = false) {
  if (!L || !S || !T) return set_error(h, FR_ERR_INVALID_ARG, "null descriptor");
  std::memset(it, 0, sizeof *it);
  if (!L->ctrl_z) return set_error(h, FR_ERR_INVALID_ARG, "lens.ctrl_z is null");
  if (any_degree) {
    if (L->p < 1 || L->q < 1 || L->p > 5 || L->q > 5)
      return set_error(h, FR_ERR_UNSUPPORTED, "derivative maps take degrees 1 to 5");
    if (L->n1 < L->p || L->n2 < L->q)
      return set_error(h, FR_ERR_INVALID_ARG, "a degree-p net needs at least p + 1 control points");
  } else if (L->p != 3 || L->q != 3) {
    return set_error(h, FR_ERR_UNSUPPORTED, "only degrees p = q = 3 are implemented");
  }
  if (L->n1 < 3 || L->n2 < 3 || L->n1 + 1 > fr::kMaxCtrl || L->n2 + 1 > fr::kMaxCtrl)
    return set_error(h, FR_ERR_UNSUPPORTED, "control net must be between 4x4 and %dx%d", fr::kMaxCtrl,
                     fr::kMaxCtrl);
  if (!(L->rx > 0.0f) || !(L->ry > 0.0f) || !finite(L->rx) || !finite(L->ry) || !finite(L->z_in) ||
      !(L->n_glass > 0.0f) || !finite(L->n_glass))
    return set_error(h, FR_ERR_INVALID_ARG, "lens geometry must be finite with rx, ry, n_glass > 0");
  if (n_rays == 0) return set_error(h, FR_ERR_INVALID_ARG, "n_rays must be positive");
  if (begin > n_rays) return set_error(h, FR_ERR_INVALID_ARG, "ray_begin beyond n_rays");
  if (count == UINT64_MAX) count = n_rays - begin;
  if (count > n_rays - begin) return set_error(h, FR_ERR_INVALID_ARG, "ray range beyond n_rays");
  if (S && S->kind == FR_SOURCE_POINT && count > 0xffffffffull)
    return set_error(h, FR_ERR_UNSUPPORTED, "a point-source call traces at most 2^32 - 1 rays");
  if (!(T->Rx > 0.0f) || !(T->Ry > 0.0f) || !finite(T->Rx) || !finite(T->Ry) || !finite(T->z_screen))
    return set_error(h, FR_ERR_INVALID_ARG, "screen half-widths must be positive and finite");
  if (T->nx < 1 || T->ny < 1 || T->nx > 4096 || T->ny > 4096)
    return set_error(h, FR_ERR_INVALID_ARG, "screen pixels must be 1..4096 per axis");
  if (T->nu_x != T->nu_y || T->nu_x < 1 || T->nu_x > 11 || T->nu_x % 2 == 0)
    return set_error(h, FR_ERR_UNSUPPORTED, "filter sizes must be equal and odd, 1 to 11");
  if (!(T->alpha > 0.0f) || !finite(T->alpha)) return set_error(h, FR_ERR_INVALID_ARG, "alpha must be positive");
  if (!finite(S->flux)) return set_error(h, FR_ERR_INVALID_ARG, "flux must be finite");
  // Lens.
  it->ctrl = L->ctrl_z;
  it->ncu = L->n1 + 1;
  it->ncv = L->n2 + 1;
  it->p = L->p;
  it->q = L->q;
  it->nsu = it->ncu - L->p;
  it->nsv = it->ncv - L->q;
  it->rx = L->rx;
  it->ry = L->ry;
  it->z_in = L->z_in;
  it->n_glass = L->n_glass;
  it->ku = (float)it->nsu / (2.0f * L->rx);
  it->kv = (float)it->nsv / (2.0f * L->ry);
  const double nr = (L->n_glass - 1.0) / (L->n_glass + 1.0);
  it->R0 = (float)(nr * nr);
  it->nparam = it->ncu * it->ncv;
  if (L->entry_ctrl_z) {
    if (L->entry_n1 < 3 || L->entry_n2 < 3 || L->entry_n1 + 1 > fr::kMaxCtrl || L->entry_n2 + 1 > fr::kMaxCtrl)
      return set_error(h, FR_ERR_UNSUPPORTED, "entry net must be between 4x4 and %dx%d", fr::kMaxCtrl,
                       fr::kMaxCtrl);
    if (o.mesh_nu > 0) return set_error(h, FR_ERR_UNSUPPORTED, "the triangle mesh takes a flat entry face");
    it->two_face = 1;
    it->ctrl_in = L->entry_ctrl_z;
    it->ncu_in = L->entry_n1 + 1;
    it->ncv_in = L->entry_n2 + 1;
    it->nsu_in = it->ncu_in - 3;
    it->nsv_in = it->ncv_in - 3;
    it->ku_in = (float)it->nsu_in / (2.0f * L->rx);
    it->kv_in = (float)it->nsv_in / (2.0f * L->ry);
    it->nparam += it->ncu_in * it->ncv_in;
  }
  // Source.
  it->kind = S->kind;
  it->seed = seed;
  it->n_rays = n_rays;
  it->ray_begin = begin;
  it->ray_end = begin + count;
  it->omega0 = (float)((double)S->flux / (double)n_rays);
  if (S->kind == FR_SOURCE_COLLIMATED) {
    if (S->cols < 1 || S->rows < 1 || (uint64_t)S->cols * (uint64_t)S->rows != n_rays)
      return set_error(h, FR_ERR_INVALID_ARG, "collimated source needs n_rays == cols * rows");
    if (S->cols > (1 << 24) || S->rows > (1 << 24))
      return set_error(h, FR_ERR_INVALID_ARG, "collimated grid side above 2^24");
    it->cols = S->cols;
    it->rows = S->rows;
    const uint64_t c = (uint64_t)S->cols, lo = begin, hi = begin + count;
    it->row_lo = (uint32_t)(lo / c);
    it->row_hi = hi > lo ? (uint32_t)((hi - 1) / c + 1) : it->row_lo;
    it->col_lo = (uint32_t)(lo - (uint64_t)it->row_lo * c);
    it->col_hi = hi > lo ? (uint32_t)(hi - (uint64_t)(it->row_hi - 1) * c) : 0u;
    it->jitter = S->jitter ? 1 : 0;
    it->gnx = it->gny = 1;
  } else if (S->kind == FR_SOURCE_POINT) {
    if (!(S->half_angle > 0.0f) || !(S->half_angle < 1.5707963f))
      return set_error(h, FR_ERR_INVALID_ARG, "half_angle must be in (0, pi/2)");
    if (S->grid_nx < 1 || S->grid_ny < 1 || S->grid_nx > 4096 || S->grid_ny > 4096)
      return set_error(h, FR_ERR_INVALID_ARG, "grid of sources must be 1..4096 per axis");
    const uint64_t nsrc = (uint64_t)S->grid_nx * (uint64_t)S->grid_ny;
    if (n_rays % nsrc != 0) return set_error(h, FR_ERR_INVALID_ARG, "n_rays must be a multiple of the sources");
    if (n_rays / nsrc > 0xffffffffull) return set_error(h, FR_ERR_UNSUPPORTED, "more than 2^32 rays per source");
    if (!(S->pos[2] < L->z_in) || !finite(S->pos[0]) || !finite(S->pos[1]))
      return set_error(h, FR_ERR_INVALID_ARG, "the point source must lie before the entry face");
    it->px = S->pos[0];
    it->py = S->pos[1];
    it->pz = S->pos[2];
    it->omc_max = (float)(1.0 - std::cos((double)S->half_angle));
    it->gnx = S->grid_nx;
    it->gny = S->grid_ny;
    it->gx0 = S->grid_nx > 1 ? -0.5f * S->grid_w : 0.0f;
    it->gy0 = S->grid_ny > 1 ? -0.5f * S->grid_h : 0.0f;
    it->gdx = S->grid_nx > 1 ? S->grid_w / (float)(S->grid_nx - 1) : 0.0f;
    it->gdy = S->grid_ny > 1 ? S->grid_h / (float)(S->grid_ny - 1) : 0.0f;
    it->per_src = (uint32_t)(n_rays / nsrc);
  } else {
    return set_error(h, FR_ERR_INVALID_ARG, "unknown source kind %d", S->kind);
  }
  // Screen.
  it->z_screen = T->z_screen;
  it->Rx = T->Rx;
  it->Ry = T->Ry;
  it->nx = T->nx;
  it->ny = T->ny;
  it->nu = T->nu_x;
  it->ncol = T->nx + T->nu_x - 1;
  it->nrow = T->ny + T->nu_y - 1;
  const double wx = 2.0 * T->Rx / T->nx, wy = 2.0 * T->Ry / T->ny;
  it->inv_wx = (float)(1.0 / wx);
  it->inv_wy = (float)(1.0 / wy);
  it->Rsx = (float)(T->Rx + 0.5 * (T->nu_x - 1) * wx);
  it->Rsy = (float)(T->Ry + 0.5 * (T->nu_y - 1) * wy);
  it->gx_off = (float)((T->Rx + 0.5 * (T->nu_x - 1) * wx) / wx);
  it->gy_off = (float)((T->Ry + 0.5 * (T->nu_y - 1) * wy) / wy);
  it->ax = (float)(T->alpha * 1.4426950408889634);
  it->ay = it->ax;
  it->cut = (float)std::exp(-(double)T->alpha * 0.25 * T->nu_x * T->nu_x);
  it->inv_area = (float)(1.0 / (wx * wy));
  // Fixed-point scale of E: a single contribution is at most omega0 / area.
  {
    const double cmax = std::fabs((double)S->flux) / (double)n_rays / (wx * wy);
    int e = 0;
    std::frexp(cmax > 0 ? cmax : 1.0, &e);
    it->fixE = (float)std::ldexp(1.0, 32 - e);
    it->fixP_unit = (float)(std::fabs((double)S->flux) / (wx * wy));
  }
  it->newton_max = o.newton_max_iter;
  it->newton_tol = o.newton_tol;
  if (o.mesh_nu < 0 || o.mesh_nu > 64 || o.mesh_nv < 0 || o.mesh_nv > 64 || (o.mesh_nu > 0) != (o.mesh_nv > 0))
    return set_error(h, FR_ERR_INVALID_ARG, "mesh_nu, mesh_nv must both be 0 or both 1..64");
  if (o.hist_mode < 0 || o.hist_mode > 3 || o.window_cells < 0 || o.batch_waves < 0)
    return set_error(h, FR_ERR_INVALID_ARG, "hist_mode must be 0..3, window_cells and batch_waves >= 0");
  if (o.ray_order) {
    if (it->kind != FR_SOURCE_POINT)
      return set_error(h, FR_ERR_INVALID_ARG, "ray_order applies to point sources");
    if (begin != 0 || it->ray_end != n_rays || n_rays > 0xffffffffull)
      return set_error(h, FR_ERR_INVALID_ARG, "ray_order needs a call over all rays (and n_rays < 2^32)");
    it->order = o.ray_order;
  }
  if (it->kind == FR_SOURCE_POINT && o.mesh_nu > 0) {
    it->mesh_nu = o.mesh_nu;
    it->mesh_nv = o.mesh_nv;
    it->NU = it->nsu * o.mesh_nu;
    it->NV = it->nsv * o.mesh_nv;
    it->inv_mnu = 1.0f / (float)o.mesh_nu;
    it->inv_mnv = 1.0f / (float)o.mesh_nv;
  }
  return FR_OK;
}


// The most CTAs worth launching for an item: every lane should trace at least
// `rays_per_lane` rays (options; by default 8 collimated, 4 point-source).
void schedule_item(Item* it, int warps, const fr_options& o) {
  const uint64_t count = it->ray_end - it->ray_begin;
  const int rpl = o.rays_per_lane > 0 ? std::min(o.rays_per_lane, 64)
                                      : (it->kind == FR_SOURCE_COLLIMATED ? 8 : 4);
  const uint64_t per_cta = (uint64_t)warps * 32 * (uint64_t)rpl;
  it->max_ctas = (int)std::min<uint64_t>((count + per_cta - 1) / per_cta, 1 << 20);
}

// Warps per CTA: the most the trace kernels' launch bounds allow with two
// CTAs per SM. The collimated forward takes 12 (8 deterministic with filter
// size 5), the single-lens collimated float adjoint with filter sizes 1 and 3
// takes 10, every other variant 8.
// kind: the source of a single lens with a flat entry face, -1 for a batch or
// a two-face lens. (Collimated 2048^2 rays on GB300, before the column
// lockstep: forward 61.1 us with 12 warps, 59.1 us with 14; adjoint 79.9 us
// with 8, 76.6 us with 10. The point-source adjoint at 10 warps spills and
// took 1040 us in the ray order against 1005 us at 8.)
int pick_warps(const fr_options& o, bool adjoint, int kind, bool det, int nu) {
  int cap = 8;
  if (nu > 5) cap = 8;   // the wide-filter kernels: 256 threads
  else if (!adjoint && kind == FR_SOURCE_COLLIMATED) cap = nu <= 3 ? 12 : (det ? 8 : 12);
  else if (adjoint && kind == FR_SOURCE_COLLIMATED && !det && nu <= 3) cap = 10;
  return o.warps_per_cta > 0 ? std::min(o.warps_per_cta, cap) : cap;
}

bool want_smem_hist(const Item& it, const fr_options& o, bool det) {
  const size_t hist = (size_t)it.ncol * it.nrow * (det ? 8 : 4);
  const size_t tables = fr::lens_tables_bytes(it);
  if (hist + tables > 200 * 1024) return false;
  if (o.hist_mode == 1) return false;
  if (o.hist_mode == 2) return true;
  return hist <= 100 * 1024;
}

// Float-mode forward of one point-source lens whose extended grid does not fit
// in shared memory (or hist_mode 3): a window of the grid does. Point-source
// rays come in random order, so no CTA owns a part of the screen; every CTA
// privatises the same central window, as large as shared memory allows next
// to the lens tables (or window_cells), and as square as the grid allows.
// One CTA per SM holds it.
// In a batch (budget > 0) every item whose grid does not fit takes a window
// (collimated items too), sized so that a CTA needs at most `budget` bytes:
// two CTAs of the batch kernel share an SM.
bool plan_window(Item* it, const fr_options& o, int smem_optin, size_t budget = 0) {
  if (o.deterministic || it->two_face || it->nu > 5) return false;
  if (budget == 0 && it->kind != FR_SOURCE_POINT) return false;
  if (o.hist_mode == 1 || o.hist_mode == 2) return false;
  if (o.hist_mode == 0 && want_smem_hist(*it, o, false)) return false;
  const size_t tables = fr::lens_tables_bytes(*it);
  const size_t cap = budget > 0 ? std::min(budget, (size_t)smem_optin) : (size_t)smem_optin;
  const size_t room = cap > tables + 4096 ? cap - tables - 4096 : 0;
  long cells = (long)(room / 4);
  if (o.window_cells > 0) cells = std::min<long>(cells, o.window_cells);
  if (cells < 1) return false;
  const int side = (int)std::sqrt((double)cells);
  const int w = (int)std::min<long>(it->ncol, std::max<long>(side, cells / it->nrow));
  const int hgt = (int)std::min<long>(it->nrow, cells / w);
  if (w < 1 || hgt < 1) return false;
  it->win_c0 = (it->ncol - w) / 2;
  it->win_c1 = it->win_c0 + w;
  it->win_r0 = (it->nrow - hgt) / 2;
  it->win_r1 = it->win_r0 + hgt;
  return true;
}

constexpr int kBatchWaves = 8;

// Splits `total_ctas` over the items in proportion to their estimated cost.
void assign_ctas(std::vector<Item>& items, int total_ctas) {
  double cost_sum = 0.0;
  std::vector<double> cost(items.size());
  for (size_t i = 0; i < items.size(); ++i) {
    const double rays = (double)(items[i].ray_end - items[i].ray_begin);
    cost[i] = rays * (items[i].kind == FR_SOURCE_POINT ? 3.0 : 1.0);
    cost_sum += cost[i];
  }
  int at = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    int g = items[i].max_ctas == 0 ? 0
            : std::max(1, (int)std::lround(cost_sum > 0 ? total_ctas * cost[i] / cost_sum : 1.0));
    g = std::min(g, items[i].max_ctas);
    items[i].cta_begin = at;
    items[i].cta_end = at + g;
    at += g;
  }
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Forward / adjoint over a list of items (one launch of the trace kernel).
template <int CAP>
fr_status run_trace(fr_handle* h, std::vector<Item>& items, const fr_options& o, bool adjoint,
                    cudaStream_t st) {
  if (o.ray_order && items.size() > 1)
    return set_error(h, FR_ERR_INVALID_ARG, "ray_order applies to one lens, not to a batch");
  for (auto& it : items) {
    if (it.nu > 5 && (CAP > 1 || items.size() > 1 || it.two_face))
      return set_error(h, FR_ERR_UNSUPPORTED, "filter sizes 7, 9, 11: one single-face lens per call");
    if ((it.p != 3 || it.q != 3) && (CAP > 1 || items.size() > 1 || it.two_face || it.kind != FR_SOURCE_COLLIMATED))
      return set_error(h, FR_ERR_UNSUPPORTED, "degrees other than 3: one collimated single-face lens per call");
  }
  bool det = o.deterministic != 0;
  // A point-source forward privatises a window of its grid (plan_window); in a
  // batch every item whose grid does not fit does (two CTAs per SM).
  const bool window = !adjoint && items.size() == 1 && plan_window(&items[0], o, h->smem_optin);
  std::vector<char> batch_window(items.size(), 0);
  bool any_batch_window = false;
  if (!adjoint && items.size() > 1 && !det)
    for (size_t i = 0; i < items.size(); ++i) {
      // the whole grid when it fits the two-CTA budget beside the tables, else a window
      const size_t budget = (size_t)h->smem_optin / 2 - 1024;
      const size_t full = fr::lens_tables_bytes(items[i]) + (size_t)items[i].ncol * items[i].nrow * 4;
      fr_options ob = o;
      if (ob.hist_mode == 0 && full > budget) ob.hist_mode = 3;
      batch_window[i] = plan_window(&items[i], ob, h->smem_optin, budget) ? 1 : 0;
      any_batch_window |= batch_window[i] != 0;
    }
  // Another forward whose histograms cannot live in shared memory deposits with
  // global atomics; 64-bit integer reductions there are faster than float ones,
  // so it runs the fixed-point (deterministic) kernel and converts at the end.
  if (!adjoint && !det && !window && !any_batch_window) {
    bool any_smem = false;
    for (auto& it : items) any_smem |= want_smem_hist(it, o, false);
    det = !any_smem;
  }
  // The one CTA per SM of the window form: 20 warps with filter sizes 1 and 3
  // (the kernel's launch bounds allow 640 threads there), 16 with 5; else pick_warps.
  const int win_cap = items[0].nu <= 3 ? 20 : 16;
  int warps = window ? (o.warps_per_cta > 0 ? std::min(o.warps_per_cta, win_cap) : win_cap)
                     : pick_warps(o, adjoint, items.size() == 1 && !items[0].two_face ? items[0].kind : -1,
                                  det, items[0].nu);
  if (items[0].p != 3 || items[0].q != 3) warps = std::min(warps, 8);   // the general-degree kernels: 256 threads
  // Workspace.
  size_t at = kHeaderBytes;
  std::vector<ItemWs> ws(items.size());
  for (size_t i = 0; i < items.size(); ++i) {
    ws[i] = plan(items[i], at, det && !adjoint, det && adjoint);
    at = ws[i].end;
  }
  fr_status s = ensure_workspace(h, at, st);
  if (s != FR_OK) return s;
  size_t smem = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    Item& it = items[i];
    it.Efix = reinterpret_cast<unsigned long long*>(h->ws + ws[i].efix);
    it.Pfix = reinterpret_cast<unsigned long long*>(h->ws + ws[i].pfix);
    it.gmax = reinterpret_cast<float*>(h->ws + ws[i].gmax);
    it.defer_n = reinterpret_cast<uint32_t*>(h->ws) + 2 * i;   // (item 0's also holds the pass's ticket)
    if (may_defer(it)) it.defer = reinterpret_cast<uint32_t*>(h->ws + ws[i].defer);
    schedule_item(&it, warps, o);
    if (!adjoint) it.smem_hist = (window || batch_window[i]) ? 2 : (want_smem_hist(it, o, det) ? 1 : 0);
    smem = std::max(smem, adjoint ? fr::adj_smem_bytes(it, det) : fr::fwd_smem_bytes(it, det));
  }
  // Outputs.
  for (size_t i = 0; i < items.size(); ++i) {
    Item& it = items[i];
    if (!adjoint) {
      if (det) FR_CUDA(h, cudaMemsetAsync(it.Efix, 0, (size_t)it.ncol * it.nrow * 8, st), "memset");
      else if (!o.accumulate) FR_CUDA(h, cudaMemsetAsync(it.E, 0, (size_t)it.ncol * it.nrow * 4, st), "memset");
    } else {
      if (det) {
        FR_CUDA(h, cudaMemsetAsync(it.Pfix, 0, (size_t)it.nparam * 8, st), "memset");
        cudaError_t e = fr::launch_absmax(it.dLdE, (size_t)it.ncol * it.nrow, const_cast<float*>(it.gmax), st);
        if (e != cudaSuccess) return cuda_error(h, e, "absmax kernel");
      } else if (!o.accumulate) {
        FR_CUDA(h, cudaMemsetAsync(it.dLdP, 0, (size_t)it.nparam * 4, st), "memset");
      }
    }
  }
  // Trace.
  const int threads = warps * 32;
  const bool batch = CAP > 1;
  // A batch runs in one launch: its items must share the filter size.
  for (auto& it : items)
    if (it.nu != items[0].nu)
      return set_error(h, FR_ERR_UNSUPPORTED, "the items of a batch must have the same filter size");
  const int kinds = items[0].two_face ? 4 : (items[0].kind == FR_SOURCE_COLLIMATED ? 1 : 2);
  if (batch)
    for (auto& it : items)
      if (it.two_face) return set_error(h, FR_ERR_UNSUPPORTED, "two-face lenses are traced one per call");
  const auto key = std::make_tuple((int)adjoint, (int)det, (int)batch, items[0].nu, kinds, threads, smem);
  auto found = h->occupancy.find(key);
  int occ;
  if (found != h->occupancy.end()) {
    occ = found->second;
  } else {
    occ = adjoint ? fr::adjoint_occupancy(threads, smem, det, batch, items[0].nu, kinds)
                  : fr::forward_occupancy(threads, smem, det, batch, items[0].nu, kinds);
    h->occupancy[key] = occ;
  }
  if (occ <= 0 || smem + 1024 > (size_t)h->smem_optin)
    return set_error(h, FR_ERR_UNSUPPORTED, "trace kernel does not fit on an SM (%zu B shared)", smem);
  const int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
  int total_ctas = 0;
  for (auto& it : items) total_ctas += it.max_ctas;
  if (total_ctas > 0) {
    // A batch launches eight waves: its items' CTAs take unequal times (sizes,
    // sources and nets differ), and with one wave the SMs that finish first
    // idle until the longest CTA ends (32-lens sweep step: 27.4 ms with one
    // wave and the other batch changes undone, 13.4 ms with four waves, 12.9
    // with eight, 13.0 with sixteen).
    const int waves = o.batch_waves > 0 ? std::min(o.batch_waves, 64) : kBatchWaves;
    const int want = std::max<int>(1, h->sm_count * per_sm * (items.size() > 1 ? waves : 1));
    if (items.size() == 1) {
      items[0].cta_begin = 0;
      items[0].cta_end = std::min(want, items[0].max_ctas);
    } else {
      assign_ctas(items, std::max<int>(want, (int)items.size()));
    }
    int grid = 0;
    fr::Launch<CAP> L;
    std::memset(&L, 0, sizeof L);
    L.n_items = (int)items.size();
    L.warps = warps;
    L.early_lens = adjoint && h->pdl && h->pdl_early && !det ? 1 : 0;
    for (size_t i = 0; i < items.size(); ++i) {
      L.items[i] = items[i];
      grid = std::max(grid, items[i].cta_end);
    }
    // Items without CTAs keep cta_end == cta_begin and are skipped by the lookup.
    // While capturing, external records become event nodes of the graph.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (o.event_begin || o.event_end) FR_CUDA(h, cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing");
    const unsigned int rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (o.event_begin)
      FR_CUDA(h, cudaEventRecordWithFlags((cudaEvent_t)o.event_begin, st, rec_flags), "cudaEventRecord");
    // Programmatic overlap only where the adjoint directly follows a kernel
    // (in deterministic mode it follows the max-|dL/dE| kernel: no overlap).
    cudaError_t e = adjoint ? fr::launch_adjoint<CAP>(L, grid, smem, det, st, h->pdl && !det)
                            : fr::launch_forward<CAP>(L, grid, smem, det, st,
                                                      h->pdl && h->pdl_early && !det && o.accumulate);
    if (e != cudaSuccess) return cuda_error(h, e, adjoint ? "adjoint kernel" : "forward kernel");
    // The deferred pass: the rays whose intersection the hot kernel left to
    // the march (none on most lenses: the pass then only reads its counters).
    bool any_defer = false;
    size_t tables = 0;
    for (size_t i = 0; i < items.size(); ++i) {
      any_defer |= L.items[i].defer != nullptr;
      tables = std::max(tables, fr::lens_tables_bytes(items[i]));
    }
    if (any_defer) {
      const int dgrid = std::max(1, h->sm_count * 2);
      e = adjoint ? fr::launch_adjoint_deferred<CAP>(L, dgrid, tables, det, st)
                  : fr::launch_forward_deferred<CAP>(L, dgrid, tables, det, st);
      if (e != cudaSuccess) return cuda_error(h, e, "deferred trace kernel");
    }
    if (o.event_end)
      FR_CUDA(h, cudaEventRecordWithFlags((cudaEvent_t)o.event_end, st, rec_flags), "cudaEventRecord");
  }
  // Fixed point back to float.
  if (det) {
    for (auto& it : items) {
      cudaError_t e = adjoint ? fr::launch_grad_fix_to_float(it, o.accumulate, st)
                              : fr::launch_fix_to_float(it.Efix, it.E, (size_t)it.ncol * it.nrow,
                                                        1.0f / it.fixE, o.accumulate, st);
      if (e != cudaSuccess) return cuda_error(h, e, "fixed-point conversion");
    }
  }
  return FR_OK;
}

}  // namespace

extern "C" {

int32_t fr_abi_version(void) { return FR_ABI_VERSION; }

fr_status fr_create(fr_handle** out) {
  if (!out) return set_error(nullptr, FR_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  fr_handle* h = new (std::nothrow) fr_handle();
  if (!h) return set_error(nullptr, FR_ERR_INVALID_ARG, "out of host memory");
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e == cudaSuccess) e = fr::configure_forward(h->smem_optin);
  if (e == cudaSuccess) e = fr::configure_adjoint(h->smem_optin);
  if (e == cudaSuccess) e = fr::configure_tangent(h->smem_optin);
  if (e != cudaSuccess) {
    delete h;
    return cuda_error(nullptr, e, "fr_create");
  }
  *out = h;
  return FR_OK;
}

fr_status fr_destroy(fr_handle* h) {
  if (!h) return FR_OK;
  fr_status s = FR_OK;
  if (h->ws) {
    if (cudaDeviceSynchronize() != cudaSuccess || cudaFree(h->ws) != cudaSuccess) s = FR_ERR_CUDA;
  }
  delete h;
  return s;
}

const char* fr_last_error(const fr_handle* h) {
  if (h) return h->err.c_str();
  return g_err.empty() ? "null handle" : g_err.c_str();
}

fr_status fr_trace_forward(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed, uint64_t ray_begin,
                           uint64_t ray_count, const fr_options* options, float* E_out, fr_stats* stats_out,
                           void* stream) {
  NvtxRange nvtx_range("fr_trace_forward");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  const fr_options o = defaults(options);
  if (!E_out) return set_error(h, FR_ERR_INVALID_ARG, "E_out is null");
  std::vector<Item> items(1);
  fr_status s = make_item(h, lens, source, target, n_rays, seed, ray_begin, ray_count, o, &items[0], true);
  if (s != FR_OK) return s;
  items[0].E = E_out;
  items[0].stats = stats_out;
  return run_trace<1>(h, items, o, false, as_stream(stream));
}

fr_status fr_trace_adjoint(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed, uint64_t ray_begin,
                           uint64_t ray_count, const fr_options* options, const float* dLdE, float* dLdP_out,
                           fr_stats* stats_out, void* stream) {
  NvtxRange nvtx_range("fr_trace_adjoint");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  const fr_options o = defaults(options);
  if (!dLdE || !dLdP_out) return set_error(h, FR_ERR_INVALID_ARG, "dLdE or dLdP_out is null");
  std::vector<Item> items(1);
  fr_status s = make_item(h, lens, source, target, n_rays, seed, ray_begin, ray_count, o, &items[0], true);
  if (s != FR_OK) return s;
  items[0].dLdE = dLdE;
  items[0].dLdP = dLdP_out;
  items[0].stats = stats_out;
  return run_trace<1>(h, items, o, true, as_stream(stream));
}

fr_status fr_trace_tangent(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                           const fr_target_desc* target, uint64_t n_rays, uint64_t seed, uint64_t ray_begin,
                           uint64_t ray_count, const fr_options* options, const float* dP, int32_t n_dirs,
                           float* dE_out, fr_stats* stats_out, void* stream) {
  NvtxRange nvtx_range("fr_trace_tangent");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  const fr_options o = defaults(options);
  if (!dP || !dE_out) return set_error(h, FR_ERR_INVALID_ARG, "dP or dE_out is null");
  if (n_dirs < 1 || n_dirs > 32) return set_error(h, FR_ERR_INVALID_ARG, "n_dirs must be 1..32");
  Item it;
  fr_status s = make_item(h, lens, source, target, n_rays, seed, ray_begin, ray_count, o, &it, true);
  if (s != FR_OK) return s;
  if (it.two_face) return set_error(h, FR_ERR_UNSUPPORTED, "derivative maps take a flat entry face");
  const bool general = it.p != 3 || it.q != 3;
  if (general && it.kind != FR_SOURCE_COLLIMATED)
    return set_error(h, FR_ERR_UNSUPPORTED, "degrees other than 3: derivative maps of collimated lenses");
  it.stats = stats_out;
  const cudaStream_t st = as_stream(stream);
  if (!o.accumulate)
    FR_CUDA(h, cudaMemsetAsync(dE_out, 0, (size_t)n_dirs * it.ncol * it.nrow * sizeof(float), st), "memset");
  if (general) {
    const int warps = o.warps_per_cta > 0 ? std::min(o.warps_per_cta, 8) : 8;
    schedule_item(&it, warps, o);
    it.cta_begin = 0;
    it.cta_end = std::min(std::max(1, h->sm_count * 4), it.max_ctas);
    if (it.cta_end <= 0) return FR_OK;   // no rays
    cudaError_t e = fr::launch_tangent_general(it, warps, it.cta_end, dP, n_dirs, dE_out, st);
    if (e != cudaSuccess) return cuda_error(h, e, "tangent kernel");
    return FR_OK;
  }
  const int warps = o.warps_per_cta > 0 ? std::min(o.warps_per_cta, 8) : 8;
  schedule_item(&it, warps, o);
  const size_t smem = fr::tan_smem_bytes(it);
  const auto key = std::make_tuple(2, 0, 0, it.nu, 0, warps * 32, smem);
  auto found = h->occupancy.find(key);
  int occ;
  if (found != h->occupancy.end()) {
    occ = found->second;
  } else {
    occ = fr::tangent_occupancy(warps * 32, smem, it.nu);
    h->occupancy[key] = occ;
  }
  if (occ <= 0 || smem + 1024 > (size_t)h->smem_optin)
    return set_error(h, FR_ERR_UNSUPPORTED, "tangent kernel does not fit on an SM (%zu B shared)", smem);
  const int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
  it.cta_begin = 0;
  it.cta_end = std::min(std::max(1, h->sm_count * per_sm), it.max_ctas);
  if (it.cta_end <= 0) return FR_OK;   // no rays
  cudaError_t e = fr::launch_tangent(it, warps, it.cta_end, smem, dP, n_dirs, dE_out, st);
  if (e != cudaSuccess) return cuda_error(h, e, "tangent kernel");
  return FR_OK;
}

fr_status fr_trace_debug(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source,
                         const fr_target_desc* target, uint64_t n_rays, uint64_t seed, uint64_t ray_begin,
                         uint64_t ray_count, const fr_options* options, fr_ray_record* out, void* stream) {
  NvtxRange nvtx_range("fr_trace_debug");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  const fr_options o = defaults(options);
  if (!out) return set_error(h, FR_ERR_INVALID_ARG, "out is null");
  Item it;
  fr_status s = make_item(h, lens, source, target, n_rays, seed, ray_begin, ray_count, o, &it);
  if (s != FR_OK) return s;
  cudaError_t e = fr::launch_debug(it, out, as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "debug kernel");
  return FR_OK;
}

fr_status fr_loss_l2(fr_handle* h, const float* E, const float* E_ref, int32_t nx, int32_t ny, int32_t nu_x,
                     int32_t nu_y, double* loss_out, float* dLdE_out, void* stream) {
  NvtxRange nvtx_range("fr_loss_l2");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!E || !E_ref || !loss_out || !dLdE_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || nu_x < 1 || nu_y < 1 || nu_x % 2 == 0 || nu_y % 2 == 0)
    return set_error(h, FR_ERR_INVALID_ARG, "bad grid sizes");
  cudaError_t e = fr::launch_loss_l2(E, E_ref, nx, ny, nu_x, nu_y, loss_out, dLdE_out, as_stream(stream), h->pdl);
  if (e != cudaSuccess) return cuda_error(h, e, "loss kernel");
  return FR_OK;
}

fr_status fr_adam_step(fr_handle* h, float* P, float* m, float* v, const float* g, int64_t n, float lr, float beta1,
                       float beta2, float eps, int32_t* step, void* stream) {
  NvtxRange nvtx_range("fr_adam_step");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!P || !m || !v || !g || !step) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  if (n < 0) return set_error(h, FR_ERR_INVALID_ARG, "n < 0");
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) || !finite(lr))
    return set_error(h, FR_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
  cudaError_t e = fr::launch_adam(P, m, v, g, n, lr, beta1, beta2, eps, step, as_stream(stream), h->pdl);
  if (e != cudaSuccess) return cuda_error(h, e, "adam kernel");
  return FR_OK;
}

fr_status fr_loss_frobenius(fr_handle* h, const float* E, const float* E_ref, int32_t nx, int32_t ny, int32_t nu_x,
                            int32_t nu_y, double* loss_out, float* dLdE_out, void* stream) {
  NvtxRange nvtx_range("fr_loss_frobenius");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!E || !E_ref || !loss_out || !dLdE_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || nu_x < 1 || nu_y < 1 || nu_x % 2 == 0 || nu_y % 2 == 0)
    return set_error(h, FR_ERR_INVALID_ARG, "bad grid sizes");
  cudaError_t e =
      fr::launch_loss_frobenius(E, E_ref, nx, ny, nu_x, nu_y, loss_out, dLdE_out, as_stream(stream), h->pdl);
  if (e != cudaSuccess) return cuda_error(h, e, "Frobenius loss kernel");
  return FR_OK;
}

static fr_status check_range(fr_handle* h, int64_t n, float z_min, float z_max) {
  if (n < 0) return set_error(h, FR_ERR_INVALID_ARG, "n < 0");
  if (!finite(z_min) || !finite(z_max) || !(z_min < z_max))
    return set_error(h, FR_ERR_INVALID_ARG, "need finite z_min < z_max");
  return FR_OK;
}

fr_status fr_reparam_tanh(fr_handle* h, const float* theta, const float* offset, int64_t n, float z_min,
                          float z_max, float* P_out, void* stream) {
  NvtxRange nvtx_range("fr_reparam_tanh");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!theta || !P_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  fr_status s = check_range(h, n, z_min, z_max);
  if (s != FR_OK) return s;
  cudaError_t e = fr::launch_reparam_tanh(theta, offset, n, z_min, z_max, P_out, as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "reparametrisation kernel");
  return FR_OK;
}

fr_status fr_reparam_tanh_adjoint(fr_handle* h, const float* theta, const float* dLdP, int64_t n, float z_min,
                                  float z_max, float* dLdtheta_out, void* stream) {
  NvtxRange nvtx_range("fr_reparam_tanh_adjoint");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!theta || !dLdP || !dLdtheta_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  fr_status s = check_range(h, n, z_min, z_max);
  if (s != FR_OK) return s;
  cudaError_t e = fr::launch_reparam_tanh_adjoint(theta, dLdP, n, z_min, z_max, dLdtheta_out, as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "reparametrisation adjoint kernel");
  return FR_OK;
}

fr_status fr_offset_spherical(fr_handle* h, const fr_lens_desc* lens, float c, float R, float* offset_out,
                              void* stream) {
  NvtxRange nvtx_range("fr_offset_spherical");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!lens || !offset_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  if (lens->p != 3 || lens->q != 3) return set_error(h, FR_ERR_UNSUPPORTED, "only degrees p = q = 3");
  if (lens->n1 < 3 || lens->n2 < 3 || lens->n1 >= fr::kMaxCtrl || lens->n2 >= fr::kMaxCtrl)
    return set_error(h, FR_ERR_INVALID_ARG, "control net must be 4x4 .. %dx%d", fr::kMaxCtrl, fr::kMaxCtrl);
  if (!(lens->rx > 0.0f) || !(lens->ry > 0.0f) || !finite(lens->rx) || !finite(lens->ry) || !finite(c) ||
      !finite(R))
    return set_error(h, FR_ERR_INVALID_ARG, "bad lens size or offset parameters");
  const double rx = lens->rx, ry = lens->ry, Rd = R;
  if (Rd != 0.0 && Rd * Rd < rx * rx + ry * ry)
    return set_error(h, FR_ERR_INVALID_ARG, "sphere radius %g does not cover the control net", (double)R);
  cudaError_t e = fr::launch_offset_spherical(lens->n1, lens->n2, lens->p, lens->q, rx, ry, c, Rd, offset_out,
                                              as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "offset kernel");
  return FR_OK;
}

fr_status fr_adam_step_tanh(fr_handle* h, float* theta, float* m, float* v, const float* dLdP, const float* offset,
                            int64_t n, float lr, float beta1, float beta2, float eps, float z_min, float z_max,
                            int32_t* step, float* P_out, void* stream) {
  NvtxRange nvtx_range("fr_adam_step_tanh");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!theta || !m || !v || !dLdP || !step || !P_out) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  fr_status s = check_range(h, n, z_min, z_max);
  if (s != FR_OK) return s;
  if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) || !finite(lr))
    return set_error(h, FR_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
  cudaError_t e = fr::launch_adam_tanh(theta, m, v, dLdP, offset, n, lr, beta1, beta2, eps, z_min, z_max, step, P_out,
                                       as_stream(stream), h->pdl);
  if (e != cudaSuccess) return cuda_error(h, e, "tanh Adam kernel");
  return FR_OK;
}

static fr_status batch(fr_handle* h, const fr_batch_item* in, int32_t n_items, const fr_options* options,
                       void* stream, bool adjoint) {
  NvtxRange nvtx_range(adjoint ? "fr_trace_batch_adjoint" : "fr_trace_batch_forward");
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!in || n_items < 1 || n_items > fr::kMaxItems)
    return set_error(h, FR_ERR_INVALID_ARG, "n_items must be 1..%d", fr::kMaxItems);
  const fr_options o = defaults(options);
  std::vector<Item> items(n_items);
  for (int i = 0; i < n_items; ++i) {
    fr_status s = make_item(h, &in[i].lens, &in[i].source, &in[i].target, in[i].n_rays, in[i].seed, 0,
                            UINT64_MAX, o, &items[i]);
    if (s != FR_OK) {
      const std::string msg = h->err;
      return set_error(h, s, "item %d: %s", i, msg.c_str());
    }
    if (adjoint ? (!in[i].dLdE || !in[i].dLdP) : !in[i].E)
      return set_error(h, FR_ERR_INVALID_ARG, "item %d: null buffer", i);
    items[i].E = in[i].E;
    items[i].dLdE = in[i].dLdE;
    items[i].dLdP = in[i].dLdP;
    items[i].stats = in[i].stats;
    if (in[i].ray_order) {
      if (items[i].kind != FR_SOURCE_POINT || in[i].n_rays > 0xffffffffull)
        return set_error(h, FR_ERR_INVALID_ARG, "item %d: ray_order applies to point sources (n_rays < 2^32)", i);
      items[i].order = in[i].ray_order;
    }
  }
  return run_trace<fr::kMaxItems>(h, items, o, adjoint, as_stream(stream));
}

fr_status fr_trace_batch_forward(fr_handle* h, const fr_batch_item* items, int32_t n_items,
                                 const fr_options* options, void* stream) {
  return batch(h, items, n_items, options, stream, false);
}

fr_status fr_trace_batch_adjoint(fr_handle* h, const fr_batch_item* items, int32_t n_items,
                                 const fr_options* options, void* stream) {
  return batch(h, items, n_items, options, stream, true);
}

fr_status fr_set_programmatic_launch(fr_handle* h, int32_t enable) {
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (enable < 0 || enable > 2) return set_error(h, FR_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
  h->pdl = enable != 0;
  h->pdl_early = enable == 2;
  return FR_OK;
}

fr_status fr_zero_list(fr_handle* h, void* const* ptrs, const uint64_t* bytes, int32_t n, void* stream) {
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (n < 0 || n > fr::kMaxZero) return set_error(h, FR_ERR_INVALID_ARG, "n must be 0..%d", fr::kMaxZero);
  if (n > 0 && (!ptrs || !bytes)) return set_error(h, FR_ERR_INVALID_ARG, "null list");
  fr::ZeroList z;
  std::memset(&z, 0, sizeof z);
  for (int k = 0; k < n; ++k) {
    if (!ptrs[k] && bytes[k]) return set_error(h, FR_ERR_INVALID_ARG, "buffer %d is null", k);
    z.ptr[z.n] = ptrs[k];
    z.bytes[z.n] = bytes[k];
    ++z.n;
  }
  cudaError_t e = fr::launch_zero_list(z, as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "zero kernel");
  return FR_OK;
}

fr_status fr_ray_order(fr_handle* h, const fr_lens_desc* lens, const fr_source_desc* source, uint64_t n_rays,
                       uint64_t seed, uint32_t* order_out, void* stream) {
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  NvtxRange nvtx_range("fr_ray_order");
  if (!order_out) return set_error(h, FR_ERR_INVALID_ARG, "order_out is null");
  if (!source) return set_error(h, FR_ERR_INVALID_ARG, "null descriptor");
  if (source->kind != FR_SOURCE_POINT) return set_error(h, FR_ERR_UNSUPPORTED, "ray orders are for point sources");
  if (n_rays > 0xffffffffull) return set_error(h, FR_ERR_UNSUPPORTED, "ray orders need n_rays < 2^32");
  // The order does not depend on the screen: any valid target completes the item.
  fr_target_desc t;
  std::memset(&t, 0, sizeof t);
  t.z_screen = lens ? lens->z_in + 1.0f : 1.0f;
  t.Rx = t.Ry = 1.0f;
  t.nx = t.ny = 1;
  t.nu_x = t.nu_y = 1;
  t.alpha = 1.0f;
  const fr_options o = defaults(nullptr);
  Item it;
  fr_status s = make_item(h, lens, source, &t, n_rays, seed, 0, UINT64_MAX, o, &it);
  if (s != FR_OK) return s;
  const int m = fr::ray_order_grid(it);
  const uint64_t nk = fr::ray_order_keys(it, m);
  cudaStream_t st = as_stream(stream);
  const size_t keys_at = align_up(kHeaderBytes + nk * sizeof(uint32_t));
  const size_t partial_at = align_up(keys_at + n_rays * sizeof(uint32_t));
  s = ensure_workspace(h, partial_at + fr::ray_order_scratch_words(it, m) * sizeof(uint32_t), st);
  if (s != FR_OK) return s;
  cudaError_t e = fr::launch_ray_order(it, m, reinterpret_cast<uint32_t*>(h->ws + kHeaderBytes),
                                       reinterpret_cast<uint32_t*>(h->ws + keys_at),
                                       reinterpret_cast<uint32_t*>(h->ws + partial_at), order_out, st);
  if (e != cudaSuccess) return cuda_error(h, e, "ray order kernels");
  return FR_OK;
}

fr_status fr_probe(fr_handle* h, int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float* buf,
                   int32_t n_buf, double* ops_out, void* stream) {
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (kind < 0 || kind > 7) return set_error(h, FR_ERR_INVALID_ARG, "probe kind must be 0..7");
  if (blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1)
    return set_error(h, FR_ERR_INVALID_ARG, "probe launch: 1..2^20 blocks of 32..1024 threads (multiple of 32)");
  if (!buf || !ops_out || n_buf < 4) return set_error(h, FR_ERR_INVALID_ARG, "probe buffer of >= 4 floats needed");
  if (kind == 7 && ((n_buf & 3) != 0 || ((n_buf / 4) & (n_buf / 4 - 1)) != 0))
    return set_error(h, FR_ERR_INVALID_ARG, "reduction probe: n_buf must be 4 times a power of two");
  *ops_out = fr::probe_ops(kind, blocks, threads, iters);
  cudaError_t e = fr::launch_probe(kind, blocks, threads, iters, buf, n_buf, as_stream(stream));
  if (e != cudaSuccess) return cuda_error(h, e, "probe kernel");
  return FR_OK;
}

fr_status fr_zero(fr_handle* h, void* ptr, uint64_t bytes, void* stream) {
  if (!h) return FR_ERR_INVALID_ARG;
  h->err.clear();
  if (!ptr && bytes) return set_error(h, FR_ERR_INVALID_ARG, "null pointer");
  if (bytes) FR_CUDA(h, cudaMemsetAsync(ptr, 0, bytes, as_stream(stream)), "cudaMemsetAsync");
  return FR_OK;
}

fr_status fr_stream_wait(fr_handle* h, void* stream, int32_t timeout_ms) {
  if (!h) return FR_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(as_stream(stream));
    if (e == cudaSuccess) return FR_OK;
    if (e != cudaErrorNotReady) return cuda_error(h, e, "cudaStreamQuery");
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
    if (ms.count() >= timeout_ms) return set_error(h, FR_ERR_TIMEOUT, "stream not done after %d ms", timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fr_trace_forward_static: the forward trace with its scratch memory in one
// static device array instead of the handle's workspace.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 1u << 20;
// Cells of the largest extended grid whose int64 accumulator the array holds
// (8 bytes a cell, with room for the alignment of the plan).
constexpr int kStaticMaxFixCells = 122000;
constexpr int kStaticMaxDevices = 64;

// The scratch of fr_trace_forward_static. In host code this name is only a
// stand-in for the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_static_scratch on this device
  int sm_count = 0;
  int smem_optin = 0;
};

std::mutex g_static_mu;
StaticDevice g_static_dev[kStaticMaxDevices];

// Once per device, with that device current.
fr_status static_setup(StaticDevice** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kStaticMaxDevices)
    return set_error(nullptr, FR_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, kStaticMaxDevices);
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDevice& d = g_static_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaGetSymbolAddress(static scratch)");
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = fr::configure_forward(d.smem_optin);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "static trace set-up");
    d.scratch = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return FR_OK;
}

}  // namespace

extern "C" fr_status fr_trace_forward_static(const fr_lens_desc* lens, const fr_source_desc* source,
                                             const fr_target_desc* target, uint64_t n_rays, uint64_t seed,
                                             uint64_t ray_begin, uint64_t ray_count, const fr_options* options,
                                             float* E_out, fr_stats* stats_out, void* stream) {
  NvtxRange nvtx_range("fr_trace_forward_static");
  g_err.clear();
  const fr_options o = defaults(options);
  if (!E_out) return set_error(nullptr, FR_ERR_INVALID_ARG, "E_out is null");
  Item it;
  fr_status s = make_item(nullptr, lens, source, target, n_rays, seed, ray_begin, ray_count, o, &it);
  if (s != FR_OK) return s;
  if (it.nu > 5) return set_error(nullptr, FR_ERR_UNSUPPORTED, "filter sizes 1, 3, 5");
  StaticDevice* dev = nullptr;
  s = static_setup(&dev);
  if (s != FR_OK) return s;
  const int cells = it.ncol * it.nrow;
  bool det = o.deterministic != 0;
  if (det && cells > kStaticMaxFixCells)
    return set_error(nullptr, FR_ERR_WORKSPACE,
                     "deterministic mode: the extended grid has %d cells, the static scratch holds at most %d",
                     cells, kStaticMaxFixCells);
  // The schedule of fr_trace_forward (run_trace): a point-source grid that
  // does not fit in shared memory takes the window form; any other such grid
  // the fixed-point kernel, here while its accumulator fits the static array
  // (beyond that, float atomics: the same sums in another rounding order).
  const bool window = plan_window(&it, o, dev->smem_optin);
  if (!det && !window && !want_smem_hist(it, o, false) && cells <= kStaticMaxFixCells) det = true;
  const ItemWs w = plan(it, 0, det, false);
  if (w.end > kStaticScratchBytes)
    return set_error(nullptr, FR_ERR_WORKSPACE, "the problem needs %zu bytes of scratch, more than the %zu of the "
                     "static array", w.end, kStaticScratchBytes);
  cudaStream_t st = as_stream(stream);
  unsigned char* base = dev->scratch;
  it.Efix = reinterpret_cast<unsigned long long*>(base + w.efix);
  it.E = E_out;
  it.stats = stats_out;
  const int win_cap = it.nu <= 3 ? 20 : 16;
  const int warps = window ? (o.warps_per_cta > 0 ? std::min(o.warps_per_cta, win_cap) : win_cap)
                           : pick_warps(o, false, it.two_face ? -1 : it.kind, det, it.nu);
  schedule_item(&it, warps, o);
  it.smem_hist = window ? 2 : (want_smem_hist(it, o, det) ? 1 : 0);
  const size_t smem = fr::fwd_smem_bytes(it, det);
  cudaError_t e = cudaSuccess;
  if (det) e = cudaMemsetAsync(it.Efix, 0, (size_t)cells * 8, st);
  else if (!o.accumulate) e = cudaMemsetAsync(it.E, 0, (size_t)cells * 4, st);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaMemsetAsync");
  if (it.max_ctas > 0) {
    // point sources march in the kernel: no deferred list (its worst case
    // would not fit the static array)
    const int kinds = it.two_face ? 4 : (it.kind == FR_SOURCE_COLLIMATED ? 1 : 8);
    const int occ = fr::forward_occupancy(warps * 32, smem, det, false, it.nu, kinds);
    if (occ <= 0 || smem + 1024 > (size_t)dev->smem_optin)
      return set_error(nullptr, FR_ERR_UNSUPPORTED, "trace kernel does not fit on an SM (%zu B shared)", smem);
    const int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
    it.cta_begin = 0;
    it.cta_end = std::min(std::max(1, dev->sm_count * per_sm), it.max_ctas);
    fr::Launch<1> L;
    std::memset(&L, 0, sizeof L);
    L.n_items = 1;
    L.warps = warps;
    L.items[0] = it;
    e = fr::launch_forward<1>(L, it.cta_end, smem, det, st, false, true);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "forward kernel");
  }
  if (det) {
    e = fr::launch_fix_to_float(it.Efix, it.E, (size_t)cells, 1.0f / it.fixE, o.accumulate, st);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "fixed-point conversion");
  }
  return FR_OK;
}
