"""Synthetic initial states on the library's own Gauss-Legendre nodes.

Node coordinates come from sdg_nodes (the library); field values come from
the seeded closed-form generators of `sdg_inputs`.  Layout: the element-major
field layout of include/sdg.h, as numpy arrays of shape
(Ny, Nx, n1, n1) in 2D and (Nz, Ny, Nx, n1, n1, n1) in 3D.
"""
from __future__ import annotations

import math

import numpy as np

import sdg_inputs as si

from . import sdg

TWO_PI = 2.0 * math.pi


def coords(dim, n, L, N, dual_dir=None):
    """Physical coordinates (x, y[, z]) of every node of a main-grid field
    (dual_dir None) or of the dual grid shifted by +1/2 along dual_dir.
    Main cell i spans [i dx, (i+1) dx]; dual cell i+1/2 spans
    [(i+1/2) dx, (i+3/2) dx]."""
    xi, _ = sdg.sdg_nodes(N)
    n1 = N + 1
    shape = tuple(reversed(n[:dim])) + (n1,) * dim
    out = []
    for d in range(dim):
        dx = L[d] / n[d]
        off = 0.5 if dual_dir == d else 0.0
        c = (np.arange(n[d])[:, None] + off + xi[None, :]) * dx
        shp = [1] * (2 * dim)
        shp[dim - 1 - d] = n[d]
        shp[2 * dim - 1 - d] = n1
        out.append(np.broadcast_to(c.reshape(shp), shape))
    return tuple(out)


def taylor_green_state(dim, n, L, N, nu=0.0, t=0.0, modes=None):
    """(U list, P) of the 2D Taylor-Green vortex (plus an optional stream
    function perturbation) or of the 3D Taylor-Green initial field.  Point
    values at the nodes of each field's own grid.  P is not gauged."""
    U = []
    if dim == 2:
        for d in range(2):
            x, y = coords(2, n, L, N, d)
            v = si.taylor_green_2d(x, y, t, nu)[d]
            if modes is not None:
                v = v + si.perturbation_velocity(modes, x, y)[d]
            U.append(np.ascontiguousarray(v))
        x, y = coords(2, n, L, N)
        P = np.ascontiguousarray(si.taylor_green_2d(x, y, t, nu)[2])
    else:
        for d in range(3):
            c = coords(3, n, L, N, d)
            U.append(np.ascontiguousarray(si.taylor_green_3d(*c)[d]))
        c = coords(3, n, L, N)
        P = np.ascontiguousarray(si.taylor_green_3d(*c)[3])
    return U, P


# Workloads shaped like the configurations the method is measured on.
WORKLOADS = {
    # 2D periodic [0,2pi]^2, 8x8 cells, N=3, TG, nu=0.1, theta=0.51, dt=0.01, 10 steps
    "tg2d_8x8_N3": dict(dim=2, n=(8, 8), N=3, nu=0.1, theta=0.51, dt=0.01, steps=10, modes=None),
    # 2D 256x256, N=7, TG + 32-mode perturbation (seed 0, k<=8, amp 1e-2),
    # nu=1e-3, theta=0.51, dt=2e-3, 200 steps
    "tg2d_256x256_N7": dict(dim=2, n=(256, 256), N=7, nu=1e-3, theta=0.51, dt=2e-3, steps=200,
                            modes=dict(seed=0, nmodes=32, kmax=8, amplitude=1e-2)),
    # 3D periodic [0,2pi]^3, 48^3 cells, N=4, 3D TG, nu=1/1600, dt=1e-3, 100 steps
    "tg3d_48_N4": dict(dim=3, n=(48, 48, 48), N=4, nu=1.0 / 1600, theta=0.51, dt=1e-3, steps=100,
                       modes=None),
    # 2D 64x64, N=5, TG + 16-mode perturbation (seed 1, amp 0.05), nu=0.01, dt=5e-3, 20 steps
    "tg2d_64x64_N5": dict(dim=2, n=(64, 64), N=5, nu=0.01, theta=0.51, dt=5e-3, steps=20,
                          modes=dict(seed=1, nmodes=16, kmax=8, amplitude=0.05)),
}


def cfl_number(dim, n, L, N, dt, umax):
    """CFL number of a time step dt by Eq. CFL1:
    dt (2N+1) sum_d umax_d / dx_d, umax_d the largest |u_d|."""
    return dt * (2 * N + 1) * sum(umax[d] * n[d] / L[d] for d in range(dim))


def convection_substeps(cfl, target=0.5):
    """SSP-RK3 sub-steps that bring the explicit convection to CFL <= target."""
    return max(1, int(math.ceil(cfl / target - 1e-12)))


def workload_state(name, n_override=None):
    """(params, U, P) of a named workload; `n_override` shrinks the grid.
    params gains "L", "cfl" (Eq. CFL1 from the initial velocity) and "nsub"
    (convection sub-steps per dt that keep each explicit sub-step at
    CFL <= 0.5; 1 when dt is within the limit)."""
    w = dict(WORKLOADS[name])
    if n_override is not None:
        w["n"] = tuple(n_override)
    dim = w["dim"]
    L = (TWO_PI,) * dim
    modes = None
    if w["modes"] is not None:
        m = w["modes"]
        modes = si.stream_modes(m["seed"], m["nmodes"], m["kmax"], m["amplitude"])
    U, P = taylor_green_state(dim, w["n"], L, w["N"], modes=modes)
    w["L"] = L
    umax = [float(np.abs(u).max()) for u in U]
    w["cfl"] = cfl_number(dim, w["n"], L, w["N"], w["dt"], umax)
    w["nsub"] = convection_substeps(w["cfl"]) if w["cfl"] >= 1.0 else 1
    return w, U, P


# Batched workload: 48 independent 2D problems (seed 2): cells per side from
# {16, 32, 64, 128}, N in 2..11, nu log-uniform in [1e-4, 1e-1]; each one
# Taylor-Green plus an 8-mode perturbation (amplitude 1e-2, member i seeded
# with 1000 * seed + i), theta = 0.51, dt = 1e-3, 50 steps.
BATCH = dict(seed=2, count=48, theta=0.51, dt=1e-3, steps=50, nmodes=8, kmax=8, amplitude=1e-2)


def batch_workload(seed=None, count=None):
    """(params, problems, states): problems[i] = (2, (c, c), L, N, nu) and
    states[i] = (U list, P) of member i, with params["nsub"][i] its
    convection sub-steps (1 unless dt exceeds the limit of Eq. CFL1)."""
    w = dict(BATCH)
    if seed is not None:
        w["seed"] = seed
    if count is not None:
        w["count"] = count
    L = (TWO_PI, TWO_PI)
    problems, states, nsub = [], [], []
    for i, m in enumerate(si.batch_members(w["seed"], w["count"])):
        n = (m.cells, m.cells)
        modes = si.stream_modes(1000 * w["seed"] + i, w["nmodes"], w["kmax"], w["amplitude"])
        U, P = taylor_green_state(2, n, L, m.N, modes=modes)
        cfl = cfl_number(2, n, L, m.N, w["dt"], [float(np.abs(u).max()) for u in U])
        problems.append((2, n, L, m.N, m.nu))
        states.append((U, P))
        nsub.append(convection_substeps(cfl) if cfl >= 1.0 else 1)
    w["nsub"] = nsub
    return w, problems, states
