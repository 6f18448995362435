"""Seeded synthetic workloads for the freeform-lens trace.

This module only draws and packages inputs: control heights, target images,
source and screen geometry. It holds none of the tracing arithmetic, so that the
CUDA path and the FP64 oracle can both be fed from it without sharing any part
of the method.

The paper optimises towards images that are not available here (a circular top
hat, the TU Delft flame and a faceted ball, Sec. 3.2-3.3). Seeded smooth
Gaussian-mixture targets stand in for them, at the same order of resolution.

A workload is a plain dict::

    {"name": str,
     "lens":   {"n1", "n2", "p", "q", "P" (float64 (n1+1, n2+1)), "rx", "ry",
                "z_in", "n_glass"},
     "source": {"kind": "collimated", "cols", "rows", "jitter", "flux"}
            or {"kind": "point", "pos", "half_angle", "grid", "grid_size", "flux"},
     "n_rays": int, "seed": int,
     "target": {"z_screen", "Rx", "Ry", "nx", "ny", "nu_x", "nu_y", "alpha"},
     "E_ref": float64 (ny, nx) or None}
"""
import math

import numpy as np

# Flux of the target images: the fraction of the source flux a flat n = 1.5
# lens passes at normal incidence on both faces (two Schlick factors of 0.96).
# Only the scale of the target depends on it.
FLAT_LENS_TRANSMISSION = 0.9216


def control_heights(n_u, n_v, sigma, seed, base=0.0):
    """(n_u, n_v) heights base + N(0, sigma^2), drawn with numpy's PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return base + rng.normal(0.0, sigma, size=(n_u, n_v))


def gaussian_mixture_target(nx, ny, Rx, Ry, seed, total, components=4):
    """A smooth seeded target image on the interior nx x ny pixels.

    `components` isotropic Gaussians with means ~ U(-0.6, 0.6) R, widths
    ~ U(0.1, 0.3) R and weights ~ U(0.5, 1), evaluated at the pixel centres
    and scaled so that sum(E_ref) * pixel_area == total.
    Returns float64 (ny, nx), row j along y.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    wx, wy = 2.0 * Rx / nx, 2.0 * Ry / ny
    xs = (np.arange(nx) + 0.5) * wx - Rx
    ys = (np.arange(ny) + 0.5) * wy - Ry
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros((ny, nx))
    for _ in range(components):
        mx, my = rng.uniform(-0.6, 0.6, size=2) * (Rx, Ry)
        s = rng.uniform(0.1, 0.3) * min(Rx, Ry)
        a = rng.uniform(0.5, 1.0)
        img += a * np.exp(-((X - mx) ** 2 + (Y - my) ** 2) / (2.0 * s * s))
    return img * (total / (img.sum() * wx * wy))


def _lens(n_ctrl, sigma, seed, base, z_in):
    return {"n1": n_ctrl - 1, "n2": n_ctrl - 1, "p": 3, "q": 3,
            "P": control_heights(n_ctrl, n_ctrl, sigma, seed, base),
            "rx": 0.5, "ry": 0.5, "z_in": z_in, "n_glass": 1.5}


def with_entry_face(wl, n_ctrl, sigma, seed):
    """The workload with a freeform entry face (both faces optimised): a second
    bicubic net of n_ctrl x n_ctrl heights z_in + N(0, sigma^2) over the same
    aperture in place of the flat face z = z_in. Returns a new dict."""
    out = dict(wl)
    lens = dict(wl["lens"])
    lens["n1_in"] = lens["n2_in"] = n_ctrl - 1
    lens["P_in"] = control_heights(n_ctrl, n_ctrl, sigma, seed, lens["z_in"])
    out["lens"] = lens
    return out


def _target(z_screen, R, bins):
    return {"z_screen": z_screen, "Rx": R, "Ry": R, "nx": bins, "ny": bins,
            "nu_x": 3, "nu_y": 3, "alpha": 1.0}


def collimated(name, n_side, n_ctrl, bins, height_seed, target_seed, jitter=0,
               sigma=0.01, with_target=True):
    """Collimated beam along +z through a 1 x 1 aperture, n_side^2 rays.

    Freeform base plane z = 0, entry face z_in = -0.1, screen 5 units
    downstream over 2 x 2.
    """
    tgt = _target(5.0, 1.0, bins)
    wl = {"name": name,
          "lens": _lens(n_ctrl, sigma, height_seed, 0.0, -0.1),
          "source": {"kind": "collimated", "cols": n_side, "rows": n_side,
                     "jitter": jitter, "flux": 1.0},
          "n_rays": n_side * n_side, "seed": height_seed,
          "target": tgt, "E_ref": None}
    if with_target:
        wl["E_ref"] = gaussian_mixture_target(bins, bins, 1.0, 1.0, target_seed,
                                              FLAT_LENS_TRANSMISSION)
    return wl


# Half-width of the screen of the point-source workloads: the 30-degree cone
# through the 1 x 1 aperture of a nearly flat lens lands within +-3.2 of the
# axis on a screen 6.2 units from the source.
POINT_SCREEN_R = 3.5


def point(name, n_rays, n_ctrl, bins, height_seed, ray_seed, target_seed,
          grid=(1, 1), grid_size=(0.0, 0.0), sigma=0.01, with_target=True,
          half_angle_deg=30.0):
    """Point source (or grid of point sources) 1 unit before the entry face.

    Entry face z_in = 0, freeform heights 0.2 + N(0, sigma^2) (thickness 0.2),
    screen 5 units downstream of the freeform base plane.
    """
    tgt = _target(5.2, POINT_SCREEN_R, bins)
    wl = {"name": name,
          "lens": _lens(n_ctrl, sigma, height_seed, 0.2, 0.0),
          "source": {"kind": "point", "pos": (0.0, 0.0, -1.0),
                     "half_angle": math.radians(half_angle_deg),
                     "grid": tuple(grid), "grid_size": tuple(grid_size), "flux": 1.0},
          "n_rays": int(n_rays), "seed": ray_seed,
          "target": tgt, "E_ref": None}
    if with_target:
        # About a third of the cone's flux reaches the 1 x 1 aperture.
        wl["E_ref"] = gaussian_mixture_target(bins, bins, POINT_SCREEN_R, POINT_SCREEN_R,
                                              target_seed, 0.3)
    return wl


def wall_lens(name, n_rays, bins=32, n_ctrl=16, low=0.2, high=2.0, split=13, ray_seed=11):
    """A point source under a lens whose exit face has a step ("wall") across u:
    control heights `low` for the rows i < split and `high` from there on.

    The B-spline turns the step into a wall steeper than the glass rays, so a
    ray that meets the low part just before the wall passes under the wall and
    crosses the surface again: f(t) of the intersection (Sec. 2.2.1) has
    several roots, and the hit is the smallest one. Otherwise as `point`.
    """
    wl = point(name, n_rays, n_ctrl, bins, 1, ray_seed, 1, with_target=False)
    P = np.full((n_ctrl, n_ctrl), float(low))
    P[split:, :] = float(high)
    wl["lens"]["P"] = P
    return wl


def config(k, with_target=True):
    """The five workloads of the measurement plan, k = 1..5 (k = 5 is a list)."""
    if k == 1:
        return collimated("collimated-256x256-rays-8x8-net-32x32-bins", 256, 8, 32,
                          height_seed=1, target_seed=2, with_target=with_target)
    if k == 2:
        return collimated("collimated-2048x2048-rays-16x16-net-128x128-bins", 2048, 16, 128,
                          height_seed=3, target_seed=3, with_target=with_target)
    if k == 3:
        return point("point-16M-rays-24x24-net-256x256-bins", 1 << 24, 24, 256,
                     height_seed=4, ray_seed=4, target_seed=4, with_target=with_target)
    if k == 4:
        return point("point-grid-8x8x1M-rays-24x24-net-256x256-bins", 64 << 20, 24, 256,
                     height_seed=5, ray_seed=5, target_seed=5, grid=(8, 8),
                     grid_size=(0.2, 0.2), with_target=with_target)
    if k == 5:
        return design_sweep(32, seed=6, with_target=with_target)
    raise ValueError("configs are numbered 1..5")


def design_sweep(n_lenses, seed, with_target=True, min_rays=1 << 20, max_rays=1 << 24):
    """Independent lenses of a batched design sweep.

    Control nets from {8,12,16,24,32}^2, ray counts log-uniform in
    [min_rays, max_rays], collimated or point source with probability 1/2,
    bins from {128,192,256}^2, each with its own seeds.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_lenses):
        n_ctrl = int(rng.choice([8, 12, 16, 24, 32]))
        bins = int(rng.choice([128, 192, 256]))
        rays = int(math.exp(rng.uniform(math.log(min_rays), math.log(max_rays))))
        s = 1000 * seed + k
        if rng.uniform() < 0.5:
            side = max(1, int(round(math.sqrt(rays))))
            out.append(collimated("sweep%d-collimated" % k, side, n_ctrl, bins,
                                  height_seed=s, target_seed=s + 1, with_target=with_target))
        else:
            out.append(point("sweep%d-point" % k, rays, n_ctrl, bins, height_seed=s,
                             ray_seed=s, target_seed=s + 1, with_target=with_target))
    return out
