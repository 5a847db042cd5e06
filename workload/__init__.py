"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the bench.

This module holds problem DATA only -- configurations, seeded random numbers, the
manufactured solution and its forcing -- and none of the solver's arithmetic
(no basis functions, no geometry pull-back, no preconditioner, no Krylov method).
Both the CPU oracle and the CUDA path consume what it produces; collocation points
are computed by each side independently and passed in.

Workloads (Sec. 5 of the paper uses a quarter ring and K = I; the radii and the
forcing are not printed, so they are fixed here):
* manufactured solution u = sin(pi x) sin(pi y) [sin(pi z)] (r - r0)(r1 - r), which
  vanishes on the whole boundary of the (extruded) quarter annulus;
* its forcing f = -Lap u, derived by hand (``manufactured_f``);
* additive seeded perturbation f + sigma * max|f| * z, z ~ N(0, 1) (PCG64);
* seeded Gaussian right-hand sides;
* a batch of 256 2D problems and a Poisson request stream.
"""

import math

import numpy as np

# Named configurations (sizes are elements per direction; n = n_elem + p - 2 DOFs).
CONFIGS = {
    "2d_annulus_ne32_p3": dict(d=2, n_elem=32, ps=[3], r0=1.0, r1=2.0,
                               rhs="manufactured", sigma=0.0, seed=0),
    "3d_annulus_ne64": dict(d=3, n_elem=64, ps=[3, 4, 5], r0=1.0, r1=2.0,
                            rhs="manufactured", sigma=1e-3, seed=0),
    "3d_annulus_ne128": dict(d=3, n_elem=128, ps=[4, 5, 6], r0=1.0, r1=2.0,
                             rhs="manufactured", sigma=1e-3, seed=0),
    # Sec. 5's 3D domain: the quarter ring revolved about the axis (0,1,0) through
    # (-1,-1,-1); f = 1 (no closed-form solution is given for it) with the same perturbation
    "3d_revolved_ne64": dict(d=3, n_elem=64, ps=[3, 4, 5], r0=1.0, r1=2.0,
                             geometry="revolved", rhs="constant", sigma=1e-3, seed=0),
    # Sec. 3.2's convection-diffusion operator -Lap + w . grad on the extruded ring with
    # a constant wind (5, 5, 5); f = 1 with the same perturbation
    "3d_wind_ne64": dict(d=3, n_elem=64, ps=[3, 4, 5], r0=1.0, r1=2.0,
                         wind=(5.0, 5.0, 5.0), rhs="constant", sigma=1e-3, seed=0),
    # Sec. 2.3's weighted-quadrature Galerkin discretization on Sec. 5's revolved ring (the
    # setting of the paper's WQ tables); f = 1, its WQ load vector perturbed as above
    "3d_wq_revolved_ne64": dict(d=3, n_elem=64, ps=[3, 4, 5], r0=1.0, r1=2.0,
                                geometry="revolved", scheme="wq", rhs="wq_constant",
                                sigma=1e-3, seed=0),
}


def manufactured_u(points, r0=1.0, r1=2.0):
    """u(x) at physical points (N, d)."""
    pts = np.asarray(points, dtype=np.float64)
    x, y = pts[:, 0], pts[:, 1]
    r = np.sqrt(x * x + y * y)
    g = np.sin(np.pi * x) * np.sin(np.pi * y)
    if pts.shape[1] == 3:
        g = g * np.sin(np.pi * pts[:, 2])
    return g * (r - r0) * (r1 - r)


def manufactured_f(points, r0=1.0, r1=2.0):
    """f = -Lap u for ``manufactured_u``.

    Write u = g h with h(r) = (r - r0)(r1 - r), r = sqrt(x^2 + y^2).  Then
    Lap u = g Lap h + 2 grad g . grad h + h Lap g with
    h' = r0 + r1 - 2 r, Lap h = h'' + h'/r = -2 + h'/r, grad h = h' (x, y, 0)/r,
    Lap g = -d pi^2 g.
    """
    pts = np.asarray(points, dtype=np.float64)
    d = pts.shape[1]
    x, y = pts[:, 0], pts[:, 1]
    r = np.sqrt(x * x + y * y)
    sx, cx = np.sin(np.pi * x), np.cos(np.pi * x)
    sy, cy = np.sin(np.pi * y), np.cos(np.pi * y)
    sz = np.sin(np.pi * pts[:, 2]) if d == 3 else 1.0
    g = sx * sy * sz
    gx = np.pi * cx * sy * sz
    gy = np.pi * sx * cy * sz
    h = (r - r0) * (r1 - r)
    hp = r0 + r1 - 2.0 * r
    lap_h = -2.0 + hp / r
    lap_g = -d * np.pi ** 2 * g
    lap_u = g * lap_h + 2.0 * (hp / r) * (x * gx + y * gy) + h * lap_g
    return -lap_u


def perturb(f, sigma, seed=0):
    """Additive seeded perturbation f + sigma * max|f| * z, z ~ N(0,1) (PCG64(seed))."""
    f = np.asarray(f, dtype=np.float64)
    if sigma == 0.0:
        return f.copy()
    z = np.random.Generator(np.random.PCG64(seed)).standard_normal(f.shape[0])
    return f + sigma * np.max(np.abs(f)) * z


def gaussian_rhs(N, nrhs=1, seed=0):
    """iid N(0,1) right-hand sides, shape (nrhs, N)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((nrhs, N))


def config_rhs(name, points, p_index=0):
    """Right-hand side of a named configuration at the given physical points."""
    c = CONFIGS[name]
    if c["rhs"] == "constant":
        f = np.ones(np.asarray(points).shape[0])
    else:
        f = manufactured_f(points, c["r0"], c["r1"])
    return perturb(f, c["sigma"], c["seed"] + p_index)


def batched_problems(count=256, seed=1, nrhs=8, rhs_seed=2):
    """The batched form: ``count`` independent 2D quarter-annulus problems with
    n_elem ~ U{32..512}, p ~ U{2..6}, inner radius ~ U[0.5, 1.5], outer = inner + 1,
    each with ``nrhs`` Gaussian right-hand sides (seeded per problem)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n_elem = int(rng.integers(32, 513))
        p = int(rng.integers(2, 7))
        r0 = float(rng.uniform(0.5, 1.5))
        out.append(dict(d=2, n_elem=n_elem, p=p, r0=r0, r1=r0 + 1.0,
                        nrhs=nrhs, rhs_seed=rhs_seed * 100003 + i))
    return out


def served_requests(rate=2000.0, duration=10.0, seed=3, frac_2d=0.5,
                    ne2d=(64, 1024), ne3d=(32, 160)):
    """Poisson arrivals (exponential gaps, mean 1/rate) of mixed 2D/3D solves."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            break
        if rng.uniform() < frac_2d:
            d, n_elem, p = 2, int(rng.integers(ne2d[0], ne2d[1] + 1)), int(rng.integers(2, 7))
        else:
            d, n_elem, p = 3, int(rng.integers(ne3d[0], ne3d[1] + 1)), int(rng.integers(3, 7))
        out.append(dict(t_arrival=t, d=d, n_elem=n_elem, p=p, r0=1.0, r1=2.0,
                        rhs_seed=seed * 1000003 + i))
        i += 1
    return out


def dofs(d, n_elem, p):
    """N = (n_elem + p - 2)^d."""
    return int(math.pow(n_elem + p - 2, d))
