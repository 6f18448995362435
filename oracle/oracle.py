"""numpy front end of the FP64 CPU oracle (test infrastructure only).

Loads ``oracle/liboracle.so`` (built from ``freeray_oracle.cpp`` by
``oracle/build.py``) through ctypes and takes the plain workload dicts of
``paper_2302_12031_gb300.workloads``. Nothing here computes any part of the
method: every number comes from the C++ oracle.

Status codes of the per-ray records: 0 on screen, 1 aperture miss, 2 out of the
freeform's domain, 3 total internal reflection, 4 off screen, 5 invalid lens.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, APERTURE_MISS, OUT_OF_DOMAIN, TIR, OFF_SCREEN, INVALID = range(6)


class Problem(C.Structure):
    _fields_ = [
        ("n1", C.c_int32), ("n2", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
        ("P", C.POINTER(C.c_double)),
        ("rx", C.c_double), ("ry", C.c_double), ("z_in", C.c_double), ("n_glass", C.c_double),
        ("src_kind", C.c_int32), ("cols", C.c_int32), ("rows", C.c_int32), ("jitter", C.c_int32),
        ("src_pos", C.c_double * 3), ("half_angle", C.c_double),
        ("grid_nx", C.c_int32), ("grid_ny", C.c_int32),
        ("grid_w", C.c_double), ("grid_h", C.c_double),
        ("flux", C.c_double), ("n_rays", C.c_uint64), ("seed", C.c_uint64),
        ("z_screen", C.c_double), ("Rx", C.c_double), ("Ry", C.c_double),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nu_x", C.c_int32), ("nu_y", C.c_int32),
        ("alpha", C.c_double), ("scan_points", C.c_int32),
        ("mesh_nu", C.c_int32), ("mesh_nv", C.c_int32), ("pad_", C.c_int32),
        ("P_in", C.POINTER(C.c_double)), ("n1_in", C.c_int32), ("n2_in", C.c_int32),
    ]


class Record(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("span_i", C.c_int32), ("span_j", C.c_int32), ("pad_", C.c_int32),
        ("u", C.c_double), ("v", C.c_double),
        ("x", C.c_double), ("y", C.c_double), ("z", C.c_double),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("tx", C.c_double), ("ty", C.c_double), ("tz", C.c_double),
        ("X", C.c_double), ("Y", C.c_double), ("w", C.c_double), ("t", C.c_double),
    ]


RECORD_DTYPE = np.dtype([(name, np.int32 if ct is C.c_int32 else np.float64)
                         for name, ct in Record._fields_])


class Stats(C.Structure):
    _fields_ = [("counts", C.c_uint64 * 8)]


_lib = None


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(Problem)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.or_ray_uniforms.argtypes = [C.c_uint64, C.c_uint64, dp, dp]
        L.or_knots.argtypes = [C.c_int32, C.c_int32, dp]
        L.or_basis.argtypes = [C.c_int32, C.c_int32, C.c_double, dp, dp]
        L.or_surface.argtypes = [pp, C.c_double, C.c_double, dp]
        L.or_surface.restype = C.c_int32
        L.or_refract.argtypes = [dp, dp, C.c_double, dp, dp]
        L.or_refract.restype = C.c_int32
        L.or_schlick_transmission.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_schlick_transmission.restype = C.c_double
        L.or_filter_axis.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                     C.c_double, dp, dp]
        L.or_point_ray.argtypes = [pp, C.c_uint64, dp, dp, dp]
        L.or_point_ray.restype = C.c_int32
        L.or_trace_records.argtypes = [pp, C.c_uint64, C.c_uint64, C.POINTER(Record), C.c_int32]
        L.or_trace_records.restype = C.c_int32
        L.or_trace_forward.argtypes = [pp, C.c_uint64, C.c_uint64, dp, C.POINTER(Stats), C.c_int32]
        L.or_trace_forward.restype = C.c_int32
        L.or_trace_gradient.argtypes = [pp, C.c_uint64, C.c_uint64, dp, dp, C.c_int32]
        L.or_trace_gradient.restype = C.c_int32
        L.or_trace_tangent.argtypes = [pp, C.c_uint64, C.c_uint64, dp, C.c_int32, dp, C.c_int32]
        L.or_trace_tangent.restype = C.c_int32
        L.or_loss_l2.argtypes = [dp, dp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, dp]
        L.or_loss_l2.restype = C.c_double
        L.or_adam_step.argtypes = [dp, dp, dp, dp, C.c_int32, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int32]
        L.or_loss_frobenius.argtypes = [dp, dp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, dp]
        L.or_loss_frobenius.restype = C.c_double
        L.or_greville.argtypes = [C.c_int32, C.c_int32, dp]
        L.or_offset_spherical.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                          C.c_double, C.c_double, dp]
        L.or_offset_spherical.restype = C.c_int32
        L.or_reparam_tanh.argtypes = [dp, dp, C.c_int32, C.c_double, C.c_double, dp]
        L.or_reparam_tanh_adjoint.argtypes = [dp, dp, C.c_int32, C.c_double, C.c_double, dp]
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleProblem:
    """A workload dict translated into the oracle's C structure.

    Keeps the control-height array alive for as long as the structure is used.
    `P` overrides the workload's control heights (e.g. for finite differences).
    """

    def __init__(self, wl, P=None, scan_points=1024, P_in=None):
        lens, src, tgt = wl["lens"], wl["source"], wl["target"]
        self.P = _f64(lens["P"] if P is None else P).reshape(lens["n1"] + 1, lens["n2"] + 1)
        s = Problem()
        s.n1, s.n2, s.p, s.q = lens["n1"], lens["n2"], lens["p"], lens["q"]
        s.P = _dptr(self.P)
        s.rx, s.ry, s.z_in, s.n_glass = lens["rx"], lens["ry"], lens["z_in"], lens["n_glass"]
        if src["kind"] == "collimated":
            s.src_kind = 0
            s.cols, s.rows, s.jitter = src["cols"], src["rows"], src.get("jitter", 0)
            s.grid_nx = s.grid_ny = 1
        else:
            s.src_kind = 1
            s.src_pos[:] = src["pos"]
            s.half_angle = src["half_angle"]
            s.grid_nx, s.grid_ny = src.get("grid", (1, 1))
            s.grid_w, s.grid_h = src.get("grid_size", (0.0, 0.0))
        s.flux = src["flux"]
        s.n_rays, s.seed = wl["n_rays"], wl["seed"]
        s.z_screen, s.Rx, s.Ry = tgt["z_screen"], tgt["Rx"], tgt["Ry"]
        s.nx, s.ny, s.nu_x, s.nu_y = tgt["nx"], tgt["ny"], tgt["nu_x"], tgt["nu_y"]
        s.alpha = tgt["alpha"]
        s.scan_points = scan_points
        mesh = wl.get("mesh", (0, 0))
        s.mesh_nu, s.mesh_nv = mesh
        # optional freeform entry face; P_in overrides its heights
        self.P_in = None
        if lens.get("P_in") is not None or P_in is not None:
            self.P_in = _f64(lens["P_in"] if P_in is None else P_in).reshape(lens["n1_in"] + 1, lens["n2_in"] + 1)
            s.P_in = _dptr(self.P_in)
            s.n1_in, s.n2_in = lens["n1_in"], lens["n2_in"]
        self.s = s
        self.ext_shape = (tgt["ny"] + tgt["nu_y"] - 1, tgt["nx"] + tgt["nu_x"] - 1)

    def ptr(self):
        return C.byref(self.s)


def _range(wl, begin, count):
    if count is None:
        count = wl["n_rays"] - begin
    return int(begin), int(count)


def trace_forward(wl, P=None, begin=0, count=None, nthreads=0, P_in=None):
    """(E on the extended grid, counts per status) for rays [begin, begin+count)."""
    pb = OracleProblem(wl, P, P_in=P_in)
    begin, count = _range(wl, begin, count)
    E = np.zeros(pb.ext_shape)
    st = Stats()
    rc = lib().or_trace_forward(pb.ptr(), begin, count, _dptr(E), C.byref(st), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return E, np.array(st.counts[:], dtype=np.int64)


def trace_records(wl, P=None, begin=0, count=None, nthreads=0, P_in=None):
    """Per-ray records (structured array, fields of RECORD_DTYPE)."""
    pb = OracleProblem(wl, P, P_in=P_in)
    begin, count = _range(wl, begin, count)
    out = np.zeros(count, dtype=RECORD_DTYPE)
    rc = lib().or_trace_records(pb.ptr(), begin, count,
                                out.ctypes.data_as(C.POINTER(Record)), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return out


def trace_gradient(wl, dLdE, P=None, begin=0, count=None, nthreads=0, P_in=None):
    """dL/dP^z (shape (n1+1, n2+1)) for an upstream dL/dE on the extended grid;
    with a freeform entry face the pair (dL/dP^z exit, dL/dP^z entry)."""
    pb = OracleProblem(wl, P, P_in=P_in)
    begin, count = _range(wl, begin, count)
    g = _f64(dLdE)
    assert g.shape == pb.ext_shape
    n_out = pb.P.size
    out = np.zeros(n_out + (pb.P_in.size if pb.P_in is not None else 0))
    rc = lib().or_trace_gradient(pb.ptr(), begin, count, _dptr(g), _dptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    if pb.P_in is None:
        return out.reshape(pb.P.shape)
    return out[:n_out].reshape(pb.P.shape), out[n_out:].reshape(pb.P_in.shape)


def trace_tangent(wl, dP, P=None, begin=0, count=None, nthreads=0):
    """Directional derivatives (dE/dP^z) dP_k of the irradiance: dP of shape
    (n_dirs, n1+1, n2+1) (or one direction (n1+1, n2+1)); returns
    (n_dirs, rows, cols) extended grids (or one grid)."""
    pb = OracleProblem(wl, P)
    begin, count = _range(wl, begin, count)
    d = _f64(dP)
    if pb.P_in is None:
        single = d.ndim == 2
        if single:
            d = d[None]
        assert d.shape[1:] == pb.P.shape
    else:   # directions over the exit heights followed by the entry heights
        single = d.ndim == 1
        if single:
            d = d[None]
        assert d.shape[1] == pb.P.size + pb.P_in.size
    out = np.zeros((d.shape[0],) + pb.ext_shape)
    rc = lib().or_trace_tangent(pb.ptr(), begin, count, _dptr(d), d.shape[0], _dptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return out[0] if single else out


def loss_l2(wl, E):
    """(L, dL/dE on the extended grid) for the workload's interior target."""
    tgt = wl["target"]
    E = _f64(E)
    Eref = _f64(wl["E_ref"])
    d = np.zeros_like(E)
    L = lib().or_loss_l2(_dptr(E), _dptr(Eref), tgt["nx"], tgt["ny"], tgt["nu_x"], tgt["nu_y"], _dptr(d))
    return L, d


def loss_frobenius(wl, E, E_ref=None):
    """(L, dL/dE on the extended grid) of the paper's normalised Frobenius loss."""
    tgt = wl["target"]
    E = _f64(E)
    Eref = _f64(wl["E_ref"] if E_ref is None else E_ref)
    d = np.zeros_like(E)
    L = lib().or_loss_frobenius(_dptr(E), _dptr(Eref), tgt["nx"], tgt["ny"], tgt["nu_x"], tgt["nu_y"], _dptr(d))
    return L, d


def greville(n, p):
    out = np.zeros(n + 1)
    lib().or_greville(n, p, _dptr(out))
    return out


def offset_spherical(n1, n2, p, q, rx, ry, c, R):
    """Offsets f(P^x, P^y) at the control points, (n1+1) x (n2+1); None if the
    sphere does not cover every control point."""
    out = np.zeros((n1 + 1, n2 + 1))
    if lib().or_offset_spherical(n1, n2, p, q, rx, ry, c, R, _dptr(out)) != 0:
        return None
    return out


def reparam_tanh(theta, z_min, z_max, offset=None):
    theta = _f64(theta)
    P = np.zeros_like(theta)
    off = None if offset is None else _f64(offset)
    lib().or_reparam_tanh(_dptr(theta), None if off is None else _dptr(off), theta.size, z_min, z_max, _dptr(P))
    return P


def reparam_tanh_adjoint(theta, dLdP, z_min, z_max):
    theta = _f64(theta)
    g = _f64(dLdP)
    out = np.zeros_like(theta)
    lib().or_reparam_tanh_adjoint(_dptr(theta), _dptr(g), theta.size, z_min, z_max, _dptr(out))
    return out


def adam_step(theta, m, v, g, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().or_adam_step(_dptr(theta), _dptr(m), _dptr(v), _dptr(g), theta.size, lr, beta1, beta2, eps, step)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def ray_uniforms(seed, ray_id):
    a, b = C.c_double(), C.c_double()
    lib().or_ray_uniforms(seed, ray_id, C.byref(a), C.byref(b))
    return a.value, b.value


def knots(n, p):
    out = np.zeros(n + p + 2)
    lib().or_knots(n, p, _dptr(out))
    return out


def basis(n, p, u):
    N = np.zeros(n + 1)
    dN = np.zeros(n + 1)
    lib().or_basis(n, p, float(u), _dptr(N), _dptr(dN))
    return N, dN


def surface(wl, u, v, P=None):
    """(Z, Z_u, Z_v, Z_uu, Z_uv, Z_vv) at (u, v)."""
    pb = OracleProblem(wl, P)
    out = np.zeros(6)
    if lib().or_surface(pb.ptr(), float(u), float(v), _dptr(out)) != 0:
        raise ValueError("oracle rejected the problem")
    return out


def refract(d, n, eta):
    """(t, cos_t) or None on total internal reflection."""
    d = _f64(d); n = _f64(n)
    t = np.zeros(3)
    ct = C.c_double()
    if lib().or_refract(_dptr(d), _dptr(n), eta, _dptr(t), C.byref(ct)) != 0:
        return None
    return t, ct.value


def schlick_transmission(n1, n2, cos_low):
    return lib().or_schlick_transmission(n1, n2, cos_low)


def filter_axis(x, Rstar, w, ncell, nu, alpha):
    f = np.zeros(ncell)
    s = C.c_double()
    lib().or_filter_axis(x, Rstar, w, ncell, nu, alpha, _dptr(f), C.byref(s))
    return f, s.value


def point_ray(wl, ray_id):
    """(status, entry point o, in-glass direction d, entry transmission T1)."""
    pb = OracleProblem(wl)
    o = np.zeros(3); d = np.zeros(3); T1 = C.c_double()
    st = lib().or_point_ray(pb.ptr(), ray_id, _dptr(o), _dptr(d), C.byref(T1))
    return st, o, d, T1.value


def default_threads():
    return os.cpu_count() or 1
