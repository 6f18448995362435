"""ctypes binding of the C ABI in include/freeray.h.

The functions below carry the same names as the C entry points and only
marshal arguments: torch tensors become device pointers, the current torch
stream becomes the cudaStream_t. Every step of the trace runs in the CUDA
kernels of libfreeray.so; there is no CPU fallback. If the library is missing
the import of this module's functions fails loudly (build it with
``__graft_entry__.build()`` or ``python -m paper_2302_12031_gb300._build``).
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfreeray.so")

# fr_status
FR_OK, FR_ERR_INVALID_ARG, FR_ERR_UNSUPPORTED, FR_ERR_CUDA, FR_ERR_WORKSPACE, FR_ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "FR_OK", 1: "FR_ERR_INVALID_ARG", 2: "FR_ERR_UNSUPPORTED", 3: "FR_ERR_CUDA",
                4: "FR_ERR_WORKSPACE", 5: "FR_ERR_TIMEOUT"}
FR_SOURCE_COLLIMATED, FR_SOURCE_POINT = 0, 1
# per-ray causes (fr_stats.rays index)
RAY_CAUSES = ["on_screen", "aperture_miss", "out_of_domain", "tir", "off_screen", "invalid", "newton_fail",
              "reserved"]
ALL_RAYS = 0xFFFFFFFFFFFFFFFF


class LensDesc(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
                ("ctrl_z", C.c_void_p), ("rx", C.c_float), ("ry", C.c_float),
                ("z_in", C.c_float), ("n_glass", C.c_float),
                ("entry_ctrl_z", C.c_void_p), ("entry_n1", C.c_int32), ("entry_n2", C.c_int32)]


class SourceDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("jitter", C.c_int32), ("cols", C.c_int32), ("rows", C.c_int32),
                ("pos", C.c_float * 3), ("half_angle", C.c_float),
                ("grid_nx", C.c_int32), ("grid_ny", C.c_int32),
                ("grid_w", C.c_float), ("grid_h", C.c_float), ("flux", C.c_float)]


class TargetDesc(C.Structure):
    _fields_ = [("z_screen", C.c_float), ("Rx", C.c_float), ("Ry", C.c_float),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nu_x", C.c_int32), ("nu_y", C.c_int32),
                ("alpha", C.c_float)]


class Options(C.Structure):
    _fields_ = [("deterministic", C.c_int32), ("accumulate", C.c_int32),
                ("newton_max_iter", C.c_int32), ("newton_tol", C.c_float),
                ("warps_per_cta", C.c_int32), ("rays_per_lane", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("hist_mode", C.c_int32),
                ("event_begin", C.c_void_p), ("event_end", C.c_void_p),
                ("mesh_nu", C.c_int32), ("mesh_nv", C.c_int32), ("ray_order", C.c_void_p),
                ("window_cells", C.c_int32), ("batch_waves", C.c_int32), ("reserved", C.c_int32 * 2)]


class Stats(C.Structure):
    _fields_ = [("rays", C.c_uint64 * 8)]


class RayRecord(C.Structure):
    _fields_ = [("status", C.c_int32), ("span_i", C.c_int32), ("span_j", C.c_int32),
                ("newton_iters", C.c_int32),
                ("u", C.c_float), ("v", C.c_float), ("x", C.c_float), ("y", C.c_float), ("z", C.c_float),
                ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
                ("tx", C.c_float), ("ty", C.c_float), ("tz", C.c_float),
                ("X", C.c_float), ("Y", C.c_float), ("w", C.c_float), ("t", C.c_float)]


class BatchItem(C.Structure):
    _fields_ = [("lens", LensDesc), ("source", SourceDesc), ("target", TargetDesc),
                ("n_rays", C.c_uint64), ("seed", C.c_uint64),
                ("E", C.c_void_p), ("dLdE", C.c_void_p), ("dLdP", C.c_void_p), ("stats", C.c_void_p),
                ("ray_order", C.c_void_p)]


RECORD_FIELDS = [name for name, _ in RayRecord._fields_]

# Every symbol include/freeray.h declares, with its ctypes signature.
_SIGNATURES = {
    "fr_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "fr_destroy": (C.c_int, [C.c_void_p]),
    "fr_last_error": (C.c_char_p, [C.c_void_p]),
    "fr_abi_version": (C.c_int32, []),
    "fr_trace_forward": (C.c_int, [C.c_void_p, C.POINTER(LensDesc), C.POINTER(SourceDesc), C.POINTER(TargetDesc),
                                   C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(Options),
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_trace_adjoint": (C.c_int, [C.c_void_p, C.POINTER(LensDesc), C.POINTER(SourceDesc), C.POINTER(TargetDesc),
                                   C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(Options),
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_trace_debug": (C.c_int, [C.c_void_p, C.POINTER(LensDesc), C.POINTER(SourceDesc), C.POINTER(TargetDesc),
                                 C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(Options),
                                 C.c_void_p, C.c_void_p]),
    "fr_trace_tangent": (C.c_int, [C.c_void_p, C.POINTER(LensDesc), C.POINTER(SourceDesc), C.POINTER(TargetDesc),
                                   C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(Options),
                                   C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_loss_l2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                             C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_adam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                               C.c_float, C.c_float, C.c_float, C.c_float, C.c_void_p, C.c_void_p]),
    "fr_loss_frobenius": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_reparam_tanh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float,
                                  C.c_void_p, C.c_void_p]),
    "fr_reparam_tanh_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float,
                                          C.c_void_p, C.c_void_p]),
    "fr_offset_spherical": (C.c_int, [C.c_void_p, C.POINTER(LensDesc), C.c_float, C.c_float, C.c_void_p,
                                      C.c_void_p]),
    "fr_adam_step_tanh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_trace_batch_forward": (C.c_int, [C.c_void_p, C.POINTER(BatchItem), C.c_int32, C.POINTER(Options),
                                         C.c_void_p]),
    "fr_trace_batch_adjoint": (C.c_int, [C.c_void_p, C.POINTER(BatchItem), C.c_int32, C.POINTER(Options),
                                         C.c_void_p]),
    "fr_stream_wait": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "fr_set_programmatic_launch": (C.c_int, [C.c_void_p, C.c_int32]),
    "fr_zero": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]),
    "fr_ray_order": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p,
                               C.c_void_p]),
    "fr_zero_list": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint64), C.c_int32, C.c_void_p]),
    "fr_probe": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                           C.POINTER(C.c_double), C.c_void_p]),
    "fr_trace_forward_static": (C.c_int, [C.POINTER(LensDesc), C.POINTER(SourceDesc), C.POINTER(TargetDesc),
                                          C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(Options),
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None
ABI_VERSION = 3   # FR_ABI_VERSION of include/freeray.h: the structures' layout


def lib():
    """The loaded libfreeray.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfreeray.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.fr_abi_version() != ABI_VERSION:
            raise ImportError("%s has ABI version %d, this binding expects %d: rebuild it"
                              % (LIB_PATH, L.fr_abi_version(), ABI_VERSION))
        _lib = L
    return _lib


class FreerayError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Handle:
    """An fr_handle bound to the current CUDA device."""

    def __init__(self):
        h = C.c_void_p()
        st = lib().fr_create(C.byref(h))
        if st != FR_OK:
            raise FreerayError(st, lib().fr_last_error(None).decode())
        self.ptr = h

    def check(self, status):
        if status != FR_OK:
            raise FreerayError(status, lib().fr_last_error(self.ptr).decode())

    def close(self):
        if self.ptr:
            lib().fr_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles = {}


def default_handle(device=None):
    """One handle per device, created on first use."""
    dev = torch.cuda.current_device() if device is None else device
    h = _handles.get(dev)
    if h is None:
        with torch.cuda.device(dev):
            h = Handle()
        _handles[dev] = h
    return h


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _opts(options):
    return C.byref(options) if options is not None else None


# --- the C entry points, one to one ------------------------------------------

def fr_abi_version():
    return lib().fr_abi_version()


def fr_trace_forward(h, lens, source, target, n_rays, seed, ray_begin, ray_count, options, E_out, stats_out=None,
                     stream=None):
    h.check(lib().fr_trace_forward(h.ptr, C.byref(lens), C.byref(source), C.byref(target), n_rays, seed,
                                   ray_begin, ray_count, _opts(options), _ptr(E_out), _ptr(stats_out),
                                   _stream(stream)))


def fr_trace_adjoint(h, lens, source, target, n_rays, seed, ray_begin, ray_count, options, dLdE, dLdP_out,
                     stats_out=None, stream=None):
    h.check(lib().fr_trace_adjoint(h.ptr, C.byref(lens), C.byref(source), C.byref(target), n_rays, seed,
                                   ray_begin, ray_count, _opts(options), _ptr(dLdE), _ptr(dLdP_out),
                                   _ptr(stats_out), _stream(stream)))


def fr_trace_debug(h, lens, source, target, n_rays, seed, ray_begin, ray_count, options, out, stream=None):
    h.check(lib().fr_trace_debug(h.ptr, C.byref(lens), C.byref(source), C.byref(target), n_rays, seed,
                                 ray_begin, ray_count, _opts(options), _ptr(out), _stream(stream)))


def fr_trace_tangent(h, lens, source, target, n_rays, seed, ray_begin, ray_count, options, dP, n_dirs, dE_out,
                     stats_out=None, stream=None):
    h.check(lib().fr_trace_tangent(h.ptr, C.byref(lens), C.byref(source), C.byref(target), n_rays, seed,
                                   ray_begin, ray_count, _opts(options), _ptr(dP), n_dirs, _ptr(dE_out),
                                   _ptr(stats_out), _stream(stream)))


def fr_loss_l2(h, E, E_ref, nx, ny, nu_x, nu_y, loss_out, dLdE_out, stream=None):
    h.check(lib().fr_loss_l2(h.ptr, _ptr(E), _ptr(E_ref), nx, ny, nu_x, nu_y, _ptr(loss_out), _ptr(dLdE_out),
                             _stream(stream)))


def fr_adam_step(h, P, m, v, g, n, lr, beta1, beta2, eps, step, stream=None):
    h.check(lib().fr_adam_step(h.ptr, _ptr(P), _ptr(m), _ptr(v), _ptr(g), n, lr, beta1, beta2, eps, _ptr(step),
                               _stream(stream)))


def fr_loss_frobenius(h, E, E_ref, nx, ny, nu_x, nu_y, loss_out, dLdE_out, stream=None):
    h.check(lib().fr_loss_frobenius(h.ptr, _ptr(E), _ptr(E_ref), nx, ny, nu_x, nu_y, _ptr(loss_out),
                                    _ptr(dLdE_out), _stream(stream)))


def fr_reparam_tanh(h, theta, offset, n, z_min, z_max, P_out, stream=None):
    h.check(lib().fr_reparam_tanh(h.ptr, _ptr(theta), _ptr(offset), n, z_min, z_max, _ptr(P_out),
                                  _stream(stream)))


def fr_reparam_tanh_adjoint(h, theta, dLdP, n, z_min, z_max, dLdtheta_out, stream=None):
    h.check(lib().fr_reparam_tanh_adjoint(h.ptr, _ptr(theta), _ptr(dLdP), n, z_min, z_max, _ptr(dLdtheta_out),
                                          _stream(stream)))


def fr_offset_spherical(h, lens, c, R, offset_out, stream=None):
    h.check(lib().fr_offset_spherical(h.ptr, C.byref(lens), c, R, _ptr(offset_out), _stream(stream)))


def fr_adam_step_tanh(h, theta, m, v, dLdP, offset, n, lr, beta1, beta2, eps, z_min, z_max, step, P_out,
                      stream=None):
    h.check(lib().fr_adam_step_tanh(h.ptr, _ptr(theta), _ptr(m), _ptr(v), _ptr(dLdP), _ptr(offset), n, lr, beta1,
                                    beta2, eps, z_min, z_max, _ptr(step), _ptr(P_out), _stream(stream)))


def fr_trace_batch_forward(h, items, options=None, stream=None):
    arr = (BatchItem * len(items))(*items)
    h.check(lib().fr_trace_batch_forward(h.ptr, arr, len(items), _opts(options), _stream(stream)))


def fr_trace_batch_adjoint(h, items, options=None, stream=None):
    arr = (BatchItem * len(items))(*items)
    h.check(lib().fr_trace_batch_adjoint(h.ptr, arr, len(items), _opts(options), _stream(stream)))


def fr_set_programmatic_launch(h, mode):
    """0 off, 1 on, 2 on with the adjoint reading the lens before its wait."""
    h.check(lib().fr_set_programmatic_launch(h.ptr, int(mode)))


def fr_zero(h, t, stream=None):
    """Zero a device tensor with a memset on the stream."""
    h.check(lib().fr_zero(h.ptr, _ptr(t), t.numel() * t.element_size(), _stream(stream)))


def fr_zero_list(h, tensors, stream=None):
    """Zero several device tensors in one kernel."""
    n = len(tensors)
    ptrs = (C.c_void_p * max(n, 1))(*[t.data_ptr() for t in tensors])
    sizes = (C.c_uint64 * max(n, 1))(*[t.numel() * t.element_size() for t in tensors])
    h.check(lib().fr_zero_list(h.ptr, ptrs, sizes, n, _stream(stream)))


def fr_ray_order(h, lens, source, n_rays, seed, order_out, stream=None):
    """Coherent ray order of a point source into order_out (int32 CUDA tensor of n_rays + 1:
    the permuted ray ids, then the number of them that meet the aperture)."""
    if order_out.dtype != torch.int32 or order_out.numel() != n_rays + 1 or not order_out.is_contiguous():
        raise ValueError("order_out must be a contiguous int32 tensor of n_rays + 1 elements")
    h.check(lib().fr_ray_order(h.ptr, C.byref(lens), C.byref(source), n_rays, seed, _ptr(order_out),
                               _stream(stream)))


def fr_stream_wait(h, timeout_ms, stream=None):
    h.check(lib().fr_stream_wait(h.ptr, _stream(stream), timeout_ms))


def fr_probe(h, kind, blocks, threads, iters, buf, stream=None):
    """Launch throughput probe `kind` (see the header); returns its operation count."""
    ops = C.c_double()
    h.check(lib().fr_probe(h.ptr, kind, blocks, threads, iters, _ptr(buf), buf.numel(), C.byref(ops),
                           _stream(stream)))
    return ops.value


def fr_trace_forward_static(lens, source, target, n_rays, seed, ray_begin, ray_count, options, E_out,
                            stats_out=None, stream=None):
    """fr_trace_forward without a handle and without any allocation (see the header)."""
    st = lib().fr_trace_forward_static(C.byref(lens), C.byref(source), C.byref(target), n_rays, seed, ray_begin,
                                       ray_count, _opts(options), _ptr(E_out), _ptr(stats_out), _stream(stream))
    if st != FR_OK:
        raise FreerayError(st, lib().fr_last_error(None).decode())


# --- descriptors from a workload dict ----------------------------------------

def make_options(deterministic=False, accumulate=False, newton_max_iter=0, newton_tol=0.0, warps_per_cta=0,
                 rays_per_lane=0, ctas_per_sm=0, hist_mode=0, events=None, mesh=(0, 0), window_cells=0,
                 ray_order=None, batch_waves=0):
    """fr_options; `events` = (begin, end) torch.cuda.Event pair to time the trace kernel;
    `ray_order` = the tensor of Problem.ray_order() (the options hold a reference to it;
    copies of the structure made by ctypes do not); `window_cells` bounds the window of
    hist_mode 3."""
    o = Options()
    o.deterministic = int(deterministic)
    o.accumulate = int(accumulate)
    o.newton_max_iter = newton_max_iter
    o.newton_tol = newton_tol
    o.warps_per_cta = warps_per_cta
    o.rays_per_lane = rays_per_lane
    o.ctas_per_sm = ctas_per_sm
    o.hist_mode = hist_mode
    o.mesh_nu, o.mesh_nv = mesh
    o.window_cells = window_cells
    o.batch_waves = batch_waves
    if ray_order is not None:
        if ray_order.dtype != torch.int32 or not ray_order.is_cuda or not ray_order.is_contiguous():
            raise ValueError("ray_order must be a contiguous int32 CUDA tensor (uint32 ids)")
        o.ray_order = ray_order.data_ptr()
        o.ray_order_numel = ray_order.numel()   # checked against the problem by Problem's calls
        o.ray_order_tensor = ray_order          # the options keep the order alive while they live
    if events is not None:
        o.event_begin = events[0].cuda_event
        o.event_end = events[1].cuda_event
    return o


class Problem:
    """Descriptors of one workload with its control heights on the device.

    `wl` is a workload dict (see paper_2302_12031_gb300.workloads); `ctrl_z`
    a float32 CUDA tensor of shape (n1+1, n2+1), by default the workload's.
    """

    def __init__(self, wl, ctrl_z=None, device="cuda", entry_z=None):
        lens, src, tgt = wl["lens"], wl["source"], wl["target"]
        if ctrl_z is None:
            ctrl_z = torch.as_tensor(lens["P"], dtype=torch.float32, device=device)
        self.ctrl_z = ctrl_z.contiguous()
        assert self.ctrl_z.dtype == torch.float32 and self.ctrl_z.is_cuda
        self.lens = LensDesc(lens["n1"], lens["n2"], lens["p"], lens["q"], self.ctrl_z.data_ptr(),
                             lens["rx"], lens["ry"], lens["z_in"], lens["n_glass"])
        # optional freeform entry face: its heights follow the exit heights in dL/dP
        self.entry_z = None
        self.entry_shape = None
        if lens.get("P_in") is not None:
            if entry_z is None:
                entry_z = torch.as_tensor(lens["P_in"], dtype=torch.float32, device=device)
            self.entry_z = entry_z.contiguous()
            assert self.entry_z.dtype == torch.float32 and self.entry_z.is_cuda
            self.entry_shape = (lens["n1_in"] + 1, lens["n2_in"] + 1)
            self.lens.entry_ctrl_z = self.entry_z.data_ptr()
            self.lens.entry_n1, self.lens.entry_n2 = lens["n1_in"], lens["n2_in"]
        s = SourceDesc()
        if src["kind"] == "collimated":
            s.kind = FR_SOURCE_COLLIMATED
            s.jitter, s.cols, s.rows = src.get("jitter", 0), src["cols"], src["rows"]
            s.grid_nx = s.grid_ny = 1
        else:
            s.kind = FR_SOURCE_POINT
            s.pos[:] = src["pos"]
            s.half_angle = src["half_angle"]
            s.grid_nx, s.grid_ny = src.get("grid", (1, 1))
            s.grid_w, s.grid_h = src.get("grid_size", (0.0, 0.0))
        s.flux = src["flux"]
        self.source = s
        self.target = TargetDesc(tgt["z_screen"], tgt["Rx"], tgt["Ry"], tgt["nx"], tgt["ny"], tgt["nu_x"],
                                 tgt["nu_y"], tgt["alpha"])
        self.n_rays = int(wl["n_rays"])
        self.seed = int(wl["seed"])
        self.ext_shape = (tgt["ny"] + tgt["nu_y"] - 1, tgt["nx"] + tgt["nu_x"] - 1)
        self.ctrl_shape = (lens["n1"] + 1, lens["n2"] + 1)
        self.nx, self.ny, self.nu_x, self.nu_y = tgt["nx"], tgt["ny"], tgt["nu_x"], tgt["nu_y"]
        self.device = self.ctrl_z.device

    def check_options(self, options):
        """Refuses options whose ray order (make_options(ray_order=...)) was built for another
        number of rays: the kernels read n_rays + 1 words of it."""
        if options is not None and options.ray_order:
            n = getattr(options, "ray_order_numel", None)
            if n != self.n_rays + 1:
                raise ValueError("ray_order has %s elements, this problem needs n_rays + 1 = %d"
                                 % (n, self.n_rays + 1))

    def set_ctrl(self, ctrl_z):
        """Point the lens descriptor at another control-height tensor."""
        self.ctrl_z = ctrl_z.contiguous()
        self.lens.ctrl_z = self.ctrl_z.data_ptr()

    def batch_item(self, E=None, dLdE=None, dLdP=None, stats=None, ray_order=None):
        it = BatchItem()
        it.lens, it.source, it.target = self.lens, self.source, self.target
        it.n_rays, it.seed = self.n_rays, self.seed
        it.E = None if E is None else E.data_ptr()
        it.dLdE = None if dLdE is None else dLdE.data_ptr()
        it.dLdP = None if dLdP is None else dLdP.data_ptr()
        it.stats = None if stats is None else stats.data_ptr()
        if ray_order is not None:
            if ray_order.dtype != torch.int32 or not ray_order.is_cuda or ray_order.numel() != self.n_rays + 1:
                raise ValueError("ray_order must be the int32 CUDA tensor of Problem.ray_order()")
            it.ray_order = ray_order.data_ptr()
        return it

    # Convenience wrappers (allocate outputs with torch, then call the ABI).
    def forward(self, options=None, ray_begin=0, ray_count=ALL_RAYS, E=None, stats=None, h=None):
        h = h or default_handle()
        if E is None:
            E = torch.empty(self.ext_shape, dtype=torch.float32, device=self.device)
        self.check_options(options)
        fr_trace_forward(h, self.lens, self.source, self.target, self.n_rays, self.seed, ray_begin, ray_count,
                         options, E, stats)
        return E

    def ray_order(self, h=None):
        """fr_ray_order for this problem's point source (int32 tensor: n_rays ray ids, then
        the number H of them, first in the order, that meet the aperture)."""
        out = torch.empty(self.n_rays + 1, dtype=torch.int32, device=self.device)
        fr_ray_order(h or default_handle(), self.lens, self.source, self.n_rays, self.seed, out)
        return out

    def n_params(self):
        n = self.ctrl_shape[0] * self.ctrl_shape[1]
        return n + (self.entry_shape[0] * self.entry_shape[1] if self.entry_shape else 0)

    def adjoint(self, dLdE, options=None, ray_begin=0, ray_count=ALL_RAYS, dLdP=None, stats=None, h=None):
        """dL/dP (ctrl_shape); with a freeform entry face the pair (exit, entry)."""
        h = h or default_handle()
        if dLdP is None:
            shape = self.ctrl_shape if self.entry_shape is None else (self.n_params(),)
            dLdP = torch.empty(shape, dtype=torch.float32, device=self.device)
        self.check_options(options)
        fr_trace_adjoint(h, self.lens, self.source, self.target, self.n_rays, self.seed, ray_begin, ray_count,
                         options, dLdE.contiguous(), dLdP, stats)
        if self.entry_shape is None:
            return dLdP
        flat = dLdP.reshape(-1)
        n = self.ctrl_shape[0] * self.ctrl_shape[1]
        return flat[:n].view(self.ctrl_shape), flat[n:].view(self.entry_shape)

    def tangent(self, dP, options=None, ray_begin=0, ray_count=ALL_RAYS, dE=None, stats=None, h=None):
        """Directional derivatives (dE/dP^z) dP: dP of shape (n_dirs, n1+1, n2+1) or
        (n1+1, n2+1); returns (n_dirs,) + ext_shape (or ext_shape)."""
        h = h or default_handle()
        dP = torch.as_tensor(dP, dtype=torch.float32, device=self.device).contiguous()
        single = dP.dim() == 2
        n_dirs = 1 if single else dP.shape[0]
        if dE is None:
            dE = torch.empty((n_dirs,) + self.ext_shape, dtype=torch.float32, device=self.device)
        self.check_options(options)
        fr_trace_tangent(h, self.lens, self.source, self.target, self.n_rays, self.seed, ray_begin, ray_count,
                         options, dP, n_dirs, dE, stats)
        return dE[0] if single else dE

    def debug(self, ray_begin=0, ray_count=None, options=None, h=None):
        """Per-ray records as a dict of CPU numpy arrays (one per field)."""
        h = h or default_handle()
        if ray_count is None:
            ray_count = self.n_rays - ray_begin
        raw = torch.empty((max(1, ray_count), C.sizeof(RayRecord)), dtype=torch.uint8, device=self.device)
        self.check_options(options)
        fr_trace_debug(h, self.lens, self.source, self.target, self.n_rays, self.seed, ray_begin, ray_count,
                       options, raw)
        return records_to_numpy(raw[:ray_count].cpu().numpy())


def records_to_numpy(raw_u8):
    """Split an (n, sizeof(fr_ray_record)) uint8 array into named fields."""
    import numpy as np
    dt = np.dtype([(name, np.int32 if ct is C.c_int32 else np.float32) for name, ct in RayRecord._fields_])
    assert dt.itemsize == C.sizeof(RayRecord)
    arr = np.ascontiguousarray(raw_u8).view(dt).reshape(-1)
    return {name: arr[name].copy() for name in RECORD_FIELDS}


def new_stats(device="cuda"):
    """A zeroed fr_stats on the device (8 uint64 counters, as int64)."""
    return torch.zeros(8, dtype=torch.int64, device=device)
