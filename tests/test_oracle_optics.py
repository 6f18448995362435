"""Pins of the oracle's refraction, Schlick weights, source sampling and filter.

Refraction is checked by the invariants of Snell's law, Schlick's weights
against the exact Fresnel equations, the point source against the distribution
it must sample, and the reconstruction filter (Sec. 2.3) against its defining
properties.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2302_12031_gb300 import workloads as W


def _unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


def _fresnel_unpolarised_R(n1, n2, cos_i):
    """Exact Fresnel reflectance for unpolarised light (Fowles, Sec. 2.7)."""
    sin_i = math.sqrt(max(0.0, 1.0 - cos_i * cos_i))
    sin_t = n1 / n2 * sin_i
    if sin_t >= 1.0:
        return 1.0
    cos_t = math.sqrt(1.0 - sin_t * sin_t)
    rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t)
    rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t)
    return 0.5 * (rs * rs + rp * rp)


@pytest.mark.parametrize("eta", [1.0 / 1.5, 1.5, 1.2, 1.0])
def test_refraction_obeys_snell(oracle, eta):
    rng = np.random.default_rng(3)
    n_tir = 0
    for _ in range(400):
        n = _unit(rng.normal(size=3))
        d = _unit(rng.normal(size=3))
        if np.dot(d, n) < 0:
            d = -d
        ci = float(np.dot(d, n))
        res = oracle.refract(d, n, eta)
        sin_i = math.sqrt(max(0.0, 1 - ci * ci))
        if eta * sin_i > 1.0:
            assert res is None
            n_tir += 1
            continue
        assert res is not None
        t, ct = res
        assert abs(np.linalg.norm(t) - 1.0) < 1e-14                       # unit direction
        # tangential momentum: n_from (d x n) = n_to (t x n), with eta = n_from/n_to
        assert np.allclose(eta * np.cross(d, n), np.cross(t, n), atol=1e-14)
        assert abs(np.dot(np.cross(d, n), t)) < 1e-14                     # coplanar
        assert abs(ct - np.dot(t, n)) < 1e-14 and ct >= 0.0               # same side as d
    if eta > 1.0:
        assert n_tir > 0


@pytest.mark.parametrize("n_glass", [1.5, 1.7])
def test_schlick_transmission_close_to_exact_fresnel(oracle, n_glass):
    r0 = ((n_glass - 1.0) / (n_glass + 1.0)) ** 2
    # Exact at normal incidence from either side.
    assert abs(oracle.schlick_transmission(1.0, n_glass, 1.0) - (1.0 - _fresnel_unpolarised_R(1.0, n_glass, 1.0))) < 1e-15
    assert abs(oracle.schlick_transmission(n_glass, 1.0, 1.0) - (1.0 - r0)) < 1e-15
    # Slope zero at normal incidence (the paper notes how shallow it is there).
    h = 1e-4
    assert abs(oracle.schlick_transmission(1.0, n_glass, 1.0 - h) - oracle.schlick_transmission(1.0, n_glass, 1.0)) < 1e-15
    # Grazing incidence: nothing transmitted.
    assert abs(oracle.schlick_transmission(1.0, n_glass, 0.0)) < 1e-15
    # Within 0.04 of exact Fresnel at every air-side angle. For these indices the
    # fifth power is the only integer exponent that stays this close (the fourth
    # and sixth powers miss by more than 0.05).
    worst = 0.0
    for deg in np.linspace(0, 89, 179):
        c = math.cos(math.radians(deg))
        Tf = 1.0 - _fresnel_unpolarised_R(1.0, n_glass, c)
        worst = max(worst, abs(Tf - oracle.schlick_transmission(1.0, n_glass, c)))
    assert worst < 0.04


def test_point_source_samples_uniform_solid_angle(oracle):
    wl = W.point("p", 40000, 8, 8, 1, 21, 1, with_target=False)
    wl["lens"]["rx"] = wl["lens"]["ry"] = 1e3      # no aperture misses
    S = np.array(wl["source"]["pos"])
    cmax = math.cos(wl["source"]["half_angle"])
    cosphi, theta = [], []
    for rid in range(0, 40000, 4):
        st, o, d, T1 = oracle.point_ray(wl, rid)
        assert st == 0
        d0 = _unit(o - S)
        cosphi.append(d0[2])
        theta.append(math.atan2(d0[1], d0[0]) % (2 * math.pi))
        # Snell at the flat face: tangential components shrink by 1/n, direction unit.
        assert np.allclose(d[:2], d0[:2] / wl["lens"]["n_glass"], atol=1e-14)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-14
    cosphi = np.array(cosphi)
    assert cosphi.min() >= cmax and cosphi.max() <= 1.0
    # Uniform in solid angle <=> cos(phi) uniform on [cos phi_max, 1], theta uniform.
    assert stats.kstest((cosphi - cmax) / (1 - cmax), "uniform").pvalue > 1e-3
    assert stats.kstest(np.array(theta) / (2 * math.pi), "uniform").pvalue > 1e-3


def test_point_source_grid_positions(oracle):
    wl = W.point("g", 64 * 10, 8, 8, 1, 5, 1, grid=(8, 8), grid_size=(0.2, 0.2), with_target=False)
    wl["lens"]["rx"] = wl["lens"]["ry"] = 1e3
    seen = set()
    for rid in range(0, 640):
        st, o, d, _ = oracle.point_ray(wl, rid)
        # back-propagate the ray in air to the source plane z = -1
        d0x, d0y = d[0] * 1.5, d[1] * 1.5
        d0z = math.sqrt(1 - d0x * d0x - d0y * d0y)
        t = (o[2] - (-1.0)) / d0z
        sx, sy = o[0] - d0x * t, o[1] - d0y * t
        k = rid // 10
        assert abs(sx - (-0.1 + (k % 8) * 0.2 / 7)) < 1e-12
        assert abs(sy - (-0.1 + (k // 8) * 0.2 / 7)) < 1e-12
        seen.add((round(sx, 9), round(sy, 9)))
    assert len(seen) == 64


@pytest.mark.parametrize("nu", [1, 3, 5, 11])
@pytest.mark.parametrize("alpha", [1.0, 0.3, 4.0])
def test_reconstruction_filter_properties(oracle, nu, alpha):
    nx, R = 16, 1.0
    w = 2 * R / nx
    Rs = R + 0.5 * (nu - 1) * w
    ncell = nx + nu - 1
    rng = np.random.default_rng(nu)
    for x in np.concatenate([rng.uniform(-R, R, 200), [-R + 1e-9, R - 1e-9, 0.01]]):
        f, s = oracle.filter_axis(x, Rs, w, ncell, nu, alpha)
        F = f / s
        assert abs(F.sum() - 1.0) < 1e-14
        assert np.all(F >= 0.0)
        nz = np.nonzero(f)[0]
        assert nz.size <= nu and (nz.max() - nz.min()) < nu          # support nu cells
        i_in = int(math.floor((x + R) / w))                         # interior pixel of x
        c = (i_in + 0.5) * w - R
        ie = i_in + (nu - 1) // 2                                   # its extended index
        assert f[ie] == f.max()                                     # peak on its own pixel
        # mirror symmetry about the pixel centre
        fm, _ = oracle.filter_axis(2 * c - x, Rs, w, ncell, nu, alpha)
        assert np.allclose(fm[ie - (nu - 1) // 2: ie + (nu - 1) // 2 + 1],
                           f[ie - (nu - 1) // 2: ie + (nu - 1) // 2 + 1][::-1], atol=1e-15)
    # zero on the edge of the support
    f, _ = oracle.filter_axis(-R + 0.5 * w + 0.5 * nu * w, Rs, w, ncell, nu, alpha)
    assert f[0] == 0.0
    # a point on a pixel edge: with nu = 1 every cell is zero (open support),
    # with nu >= 3 the two pixels sharing the edge weigh the same
    f, s = oracle.filter_axis(0.0, Rs, w, ncell, nu, alpha)
    if nu == 1:
        assert s == 0.0
    else:
        h = (nu - 1) // 2
        assert f[nx // 2 - 1 + h] == f[nx // 2 + h] > 0.0


def test_box_limit_nu1_is_indicator(oracle):
    nx, R = 10, 1.0
    w = 0.2
    for x in np.linspace(-R + 1e-6, R - 1e-6, 77):
        f, s = oracle.filter_axis(x, R, w, nx, 1, 1.0)
        F = f / s
        i = int(math.floor((x + R) / w))
        assert F[i] == 1.0 and F.sum() == 1.0
