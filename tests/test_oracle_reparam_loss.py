"""Pins of the oracle's normalised Frobenius loss (Sec. 2.5, Eq. pipelineLoss),
Greville abscissae (Sec. 2.1), offsets of Table magndata and the tanh
reparametrisation of the control heights (Sec. 2.4.2)."""
import numpy as np

from paper_2302_12031_gb300 import workloads as W


def _wl(nx, ny, nu, E_ref):
    return {"target": {"nx": nx, "ny": ny, "nu_x": nu, "nu_y": nu}, "E_ref": E_ref}


def test_frobenius_worked_example(oracle):
    # I = (1, 0), I_ref = (0, 1): I^ - I^_ref = (1, -1), L = sqrt(2)/sqrt(2) = 1.
    # L(1, e) = 1/(1+e), so dL/dI_2 = -1; L(1+e, 0) = 1, so dL/dI_1 = 0.
    wl = _wl(2, 1, 1, np.array([[0.0, 1.0]]))
    L, d = oracle.loss_frobenius(wl, np.array([[1.0, 0.0]]))
    assert abs(L - 1.0) < 1e-15
    assert np.allclose(d, [[0.0, -1.0]], rtol=0, atol=1e-15)


def test_frobenius_scale_invariance_and_euler_identity(oracle):
    rng = np.random.default_rng(3)
    nx, ny, nu = 7, 5, 3
    Eref = rng.uniform(0, 1, size=(ny, nx))
    E = np.zeros((ny + 2, nx + 2))
    E[1:-1, 1:-1] = rng.uniform(0, 1, size=(ny, nx))
    E[0, :] = 5.0                                   # ghost pixels never enter the loss
    wl = _wl(nx, ny, nu, Eref)
    L, d = oracle.loss_frobenius(wl, E)
    L3, d3 = oracle.loss_frobenius(wl, 3.0 * E)
    assert L > 0 and abs(L3 - L) < 1e-15 * 10
    assert np.allclose(d3, d / 3.0, rtol=1e-12, atol=1e-18)
    assert abs(oracle.loss_frobenius(wl, E, E_ref=7.0 * Eref)[0] - L) < 1e-14
    # L is homogeneous of degree 0 in E, so sum E dL/dE = 0 (Euler)
    assert abs(np.sum(E[1:-1, 1:-1] * d[1:-1, 1:-1])) < 1e-14
    assert np.all(d[0, :] == 0) and np.all(d[-1, :] == 0) and np.all(d[:, 0] == 0) and np.all(d[:, -1] == 0)
    # equal up to a power-of-two scale: exactly zero loss and gradient
    E2 = np.zeros_like(E)
    E2[1:-1, 1:-1] = 2.0 * Eref
    L2, d2 = oracle.loss_frobenius(wl, E2)
    assert L2 == 0.0 and np.all(d2 == 0.0)


def test_frobenius_gradient_by_central_differences(oracle):
    rng = np.random.default_rng(4)
    nx, ny, nu = 6, 4, 3
    wl = _wl(nx, ny, nu, rng.uniform(0, 1, size=(ny, nx)))
    E = np.zeros((ny + 2, nx + 2))
    E[1:-1, 1:-1] = rng.uniform(0.2, 1, size=(ny, nx))
    L, d = oracle.loss_frobenius(wl, E)
    h = 1e-6
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            Ep, Em = E.copy(), E.copy()
            Ep[j, i] += h
            Em[j, i] -= h
            fd = (oracle.loss_frobenius(wl, Ep)[0] - oracle.loss_frobenius(wl, Em)[0]) / (2 * h)
            assert abs(fd - d[j, i]) < 1e-8 * max(1.0, abs(d[j, i])), (i, j, fd, d[j, i])


def test_frobenius_undefined_normalisation(oracle):
    wl = _wl(3, 3, 1, np.ones((3, 3)))
    L, d = oracle.loss_frobenius(wl, np.zeros((3, 3)))
    assert np.isnan(L) and np.all(d == 0)


def test_greville_bezier_values_and_linear_precision(oracle):
    assert np.allclose(oracle.greville(3, 3), [0, 1 / 3, 2 / 3, 1], rtol=0, atol=1e-15)
    for n in (3, 5, 11, 23):
        g = oracle.greville(n, 3)
        assert np.allclose(g + g[::-1], 1.0, rtol=0, atol=1e-15)       # symmetric knots
        assert np.all(np.diff(g) > 0)
        for u in np.linspace(0, 1, 37):
            N, _ = oracle.basis(n, 3, u)
            assert abs(np.dot(N, g) - u) < 1e-14          # sum_i N_i(u) u*_i = u (Sec. 2.1)


def test_offset_spherical_table_magndata(oracle):
    n1, n2, rx, ry = 7, 5, 0.5, 0.5
    flat = oracle.offset_spherical(n1, n2, 3, 3, rx, ry, 0.5, 0.0)
    assert np.all(flat == 0.5)
    for R in (8.0, 4.0, -4.0):
        f = oracle.offset_spherical(n1, n2, 3, 3, rx, ry, 0.5, R)
        x = (2 * oracle.greville(n1, 3) - 1) * rx
        y = (2 * oracle.greville(n2, 3) - 1) * ry
        X, Y = np.meshgrid(x, y, indexing="ij")
        # every offset lies on the sphere of radius |R| centred at (0, 0, c + R)
        assert np.allclose(X ** 2 + Y ** 2 + (f - 0.5 - R) ** 2, R * R, rtol=0, atol=1e-12)
        assert np.all(np.sign(R) * (f - 0.5) >= 0)       # the cap opens away from the apex
        # corner control point: P^x = r_x, P^y = r_y
        assert abs(f[-1, -1] - (0.5 + R - np.sign(R) * np.sqrt(R * R - rx * rx - ry * ry))) < 1e-14
    assert oracle.offset_spherical(n1, n2, 3, 3, rx, ry, 0.5, 0.6) is None     # 0.5^2+0.5^2 > 0.6^2


def test_reparam_tanh_range_midpoint_and_adjoint(oracle):
    rng = np.random.default_rng(5)
    theta = rng.normal(0, 2, size=50)
    off = rng.normal(0, 0.1, size=50)
    zmin, zmax = -0.05, 0.15
    P = oracle.reparam_tanh(theta, zmin, zmax, off)
    assert np.all(P - off > zmin) and np.all(P - off < zmax)
    assert np.allclose(oracle.reparam_tanh(np.zeros(4), zmin, zmax), 0.5 * (zmin + zmax), rtol=0, atol=1e-16)
    big = oracle.reparam_tanh(np.array([-40.0, 40.0]), zmin, zmax)
    assert abs(big[0] - zmin) < 1e-16 and abs(big[1] - zmax) < 1e-16
    s = np.sort(theta)
    assert np.all(np.diff(oracle.reparam_tanh(s, zmin, zmax)) > 0)
    g = rng.normal(size=50)
    adj = oracle.reparam_tanh_adjoint(theta, g, zmin, zmax)
    h = 1e-6
    fd = (oracle.reparam_tanh(theta + h, zmin, zmax, off) - oracle.reparam_tanh(theta - h, zmin, zmax, off)) / (2 * h)
    assert np.allclose(adj, g * fd, rtol=1e-8, atol=1e-12)


def test_frobenius_on_a_traced_image(oracle):
    # the loss of a real traced image, and its FD on a few interior pixels
    wl = W.collimated("c", 16, 6, 8, 1, 2)
    E, _ = oracle.trace_forward(wl)
    L, d = oracle.loss_frobenius(wl, E)
    assert 0 < L < 1
    h = 1e-7
    for (j, i) in ((1, 1), (4, 5), (8, 8)):
        Ep, Em = E.copy(), E.copy()
        Ep[j, i] += h
        Em[j, i] -= h
        fd = (oracle.loss_frobenius(wl, Ep)[0] - oracle.loss_frobenius(wl, Em)[0]) / (2 * h)
        assert abs(fd - d[j, i]) < 1e-6 * max(1e-3, abs(d[j, i]))
