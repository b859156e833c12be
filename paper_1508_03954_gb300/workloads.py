"""Seeded synthetic inputs shaped like the paper's workloads.

Input data only: vertex coordinates, Gaussian right-hand sides and k^2
fields.  No step of the solver is computed here; the same arrays are fed to
the CUDA library and to the CPU oracle.  Random draws use
numpy.random.default_rng(seed) in a fixed order.
"""
from __future__ import annotations

import math

import numpy as np

THETA = math.pi / 6


def coords(d, depth):
    """Vertex coordinates of level ``depth``: tuple of d arrays, numpy axis
    order (last axis = x), broadcastable to (3^depth+1)^d."""
    n = 3 ** depth
    x = np.arange(n + 1) / n
    out = []
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n + 1
        out.append(x.reshape(shape))
    return tuple(out)


def gaussian(d, depth, centre_xyz, width, amplitude=1.0):
    """amplitude * exp(-|x - c|^2 / (2 width^2)) at the vertices; centre given
    as (x, y[, z])."""
    cs = coords(d, depth)
    r2 = 0.0
    for ax in range(d):
        c = centre_xyz[d - 1 - ax]  # numpy axis ax is coordinate d-1-ax
        r2 = r2 + (cs[ax] - c) ** 2
    return amplitude * np.exp(-r2 / (2.0 * width ** 2))


def constant_k2(d, depth, k2):
    return np.full((3 ** depth + 1,) * d, float(k2))


def random_complex(d, depth, seed):
    rng = np.random.default_rng(seed)
    shape = (3 ** depth + 1,) * d
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def config1():
    """2D, depth 3, k = 4 pi, ECS in the outer 4 fine cells (w = 4/27),
    theta = pi/6, f = Gaussian at the centre of width 0.05, additive MG with
    d-linear transfer, omega = 0.6 on all levels, 30 cycles."""
    d, L = 2, 3
    return dict(d=d, depth=L, theta=THETA, layer_width=4.0 / 27.0,
                k2=constant_k2(d, L, (4 * math.pi) ** 2),
                f=gaussian(d, L, (0.5, 0.5), 0.05).astype(np.complex128),
                omega_s=0.6, cycles=30)


def config2(depth=6):
    """2D, depth 6, k = 20 pi, layer 0.1, theta = pi/6, f = sum of three
    Gaussians of width 0.02 with centres U[0.3,0.7]^2 drawn from rng(1)."""
    d = 2
    rng = np.random.default_rng(1)
    centres = rng.uniform(0.3, 0.7, size=(3, 2))
    f = sum(gaussian(d, depth, tuple(c), 0.02) for c in centres)
    return dict(d=d, depth=depth, theta=THETA, layer_width=0.1,
                k2=constant_k2(d, depth, (20 * math.pi) ** 2),
                f=f.astype(np.complex128), centres=centres)


def config3(depth=5):
    """3D, depth 5, k = 8 pi, layer 0.1, theta = pi/6, centred Gaussian of
    width 0.05."""
    d = 3
    return dict(d=d, depth=depth, theta=THETA, layer_width=0.1,
                k2=constant_k2(d, depth, (8 * math.pi) ** 2),
                f=gaussian(d, depth, (0.5, 0.5, 0.5), 0.05).astype(np.complex128))


def config4_specs(count=256):
    """Specs of the batched workload: rng(2) draws, per problem, depth in
    {4,5,6}, k in U[5,40], Gaussian centre in U[0.3,0.7]^2 (width 0.03)."""
    rng = np.random.default_rng(2)
    depths = rng.integers(4, 7, size=count)
    ks = rng.uniform(5.0, 40.0, size=count)
    centres = rng.uniform(0.3, 0.7, size=(count, 2))
    return [dict(d=2, depth=int(depths[i]), k=float(ks[i]), centre=tuple(centres[i]),
                 width=0.03, theta=THETA, layer_width=0.1) for i in range(count)]


def config4_problem(spec):
    d, L = spec["d"], spec["depth"]
    return dict(d=d, depth=L, theta=spec["theta"], layer_width=spec["layer_width"],
                k2=constant_k2(d, L, spec["k"] ** 2),
                f=gaussian(d, L, spec["centre"], spec["width"]).astype(np.complex128))


def config5(depth=6):
    """2D, depth 6, k^2 = E - V with E = (15 pi)^2 and V a sum of 4 Gaussians
    (amplitudes U[0, 0.3E], centres U[0.2,0.8]^2, width 0.05, rng(3)),
    theta = pi/6, layer 0.1."""
    d = 2
    E = (15 * math.pi) ** 2
    rng = np.random.default_rng(3)
    amps = rng.uniform(0.0, 0.3 * E, size=4)
    centres = rng.uniform(0.2, 0.8, size=(4, 2))
    V = sum(gaussian(d, depth, tuple(c), 0.05, a) for a, c in zip(amps, centres))
    return dict(d=d, depth=depth, theta=THETA, layer_width=0.1, E=E, V=V,
                k2=E - V, f=gaussian(d, depth, (0.5, 0.5), 0.05).astype(np.complex128))


def definite(cfg):
    """Companion with the same shapes and bytes but a definite shift
    k^2 -> -k^2 (the phi < 0 regime of Section 7.2)."""
    out = dict(cfg)
    out["k2"] = -np.asarray(cfg["k2"])
    return out


def circle_samples(npts=256, radius=0.35, centre=(0.5, 0.5), m=2):
    """Sample points x_q on a circle (x first) and weights g_q = e^{i m phi_q}
    of the far-field functional of the adjoint form."""
    phi = 2.0 * math.pi * np.arange(npts) / npts
    xy = np.stack([centre[0] + radius * np.cos(phi), centre[1] + radius * np.sin(phi)], axis=1)
    return xy, np.exp(1j * m * phi)


CHANNEL_OMEGA1 = 0.01 * (math.sqrt(3.0) - 1j)    # two-phase Jacobi factors (Section 7.4)
CHANNEL_OMEGA2 = -CHANNEL_OMEGA1.conjugate()


def channel(theta_interior_deg, depth=4):
    """The p = 2 channel problem of Section 7.4 (Eq. 08-gaussian): nodal
    f = chi = exp(-(125x)^2 - (125y)^2), k^2 = phi = 45^2 + 135^2 (exp(-(15x)^2)
    + exp(-(15y)^2)), homogeneous Dirichlet values on all faces, a 30 degree
    layer within 1/3 of the top and right faces (the high end of each axis)
    and every other cell rotated by the given interior angle; h = 1/81 at
    depth 4."""
    d = 2
    y, x = coords(d, depth)
    phi = 45.0 ** 2 + 135.0 ** 2 * (np.exp(-(15.0 * x) ** 2) + np.exp(-(15.0 * y) ** 2))
    chi = np.exp(-(125.0 * x) ** 2 - (125.0 * y) ** 2)
    return dict(d=d, depth=depth, theta=math.radians(30.0), layer_width=(0.0, 1.0 / 3.0),
                theta_interior=math.radians(theta_interior_deg),
                k2=np.broadcast_to(phi, (3 ** depth + 1,) * d).copy(),
                f=np.broadcast_to(chi, (3 ** depth + 1,) * d).astype(np.complex128))


def source_refinement(d, depth, centre=(0.0, 0.0, 0.0), radius=0.7, shrink=0.7):
    """Refinement flags of an adaptive grid that resolves a localised feature
    at ``centre`` (x first): a level-l cell is refined when its centre lies
    within radius * shrink^(l-1) of the feature (so each level covers a
    smaller region; levels 1..depth-1).  Input data only: the solver reads
    the flags as the mesh."""
    out = {}
    for lev in range(1, depth):
        n = 3 ** lev
        c = (np.arange(n) + 0.5) / n
        r2 = 0.0
        for ax in range(d):
            shape = [1] * d
            shape[ax] = n
            r2 = r2 + (c.reshape(shape) - centre[d - 1 - ax]) ** 2
        out[lev] = np.broadcast_to(r2 < (radius * shrink ** (lev - 1)) ** 2, (n,) * d).copy()
    return out
