"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This module holds no arithmetic of the staggered DG method: no basis, no
quadrature, no operator.  It only draws seeded random parameters and evaluates
closed-form velocity / pressure fields at coordinates the caller supplies.
Each side (oracle, GPU library) computes its own Gauss-Legendre node
coordinates and calls these functions on them.

Fields provided:
  * 2D Taylor-Green vortex (exact solution, Sec. 3.4.2),
  * 3D Taylor-Green initial field (Sec. 2.5),
  * ABC flow (exact solution, Sec. 3.4.3),
  * divergence-free random perturbations from a stream function
    psi = sum_m a_m sin(k_m . x + phi_m); velocity (d psi/dy, -d psi/dx).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "taylor_green_2d", "taylor_green_3d", "abc_flow", "abc_pressure",
    "StreamModes", "stream_modes", "perturbation_velocity",
    "BatchMember", "batch_members", "random_vector",
]


# ---------------------------------------------------------------- analytic fields
def taylor_green_2d(x, y, t=0.0, nu=0.0):
    """u = sin x cos y e^{-2 nu t}, v = -cos x sin y e^{-2 nu t},
    p = (cos 2x + cos 2y)/4 e^{-4 nu t}."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    e2 = math.exp(-2.0 * nu * t)
    u = np.sin(x) * np.cos(y) * e2
    v = -np.cos(x) * np.sin(y) * e2
    p = 0.25 * (np.cos(2.0 * x) + np.cos(2.0 * y)) * e2 * e2
    return u, v, p


def taylor_green_3d(x, y, z):
    """3D Taylor-Green initial field: u = sin x cos y cos z,
    v = -cos x sin y cos z, w = 0, p = (cos 2x + cos 2y)(cos 2z + 2)/16."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros(np.broadcast(x, y, z).shape)
    p = (np.cos(2.0 * x) + np.cos(2.0 * y)) * (np.cos(2.0 * z) + 2.0) / 16.0
    return u, v, w, p


def abc_flow(x, y, z, t=0.0, nu=0.0):
    """Arnold-Beltrami-Childress flow with A = B = C = 1:
    u = (sin z + cos y) e^{-nu t}, v = (sin x + cos z) e^{-nu t},
    w = (sin y + cos x) e^{-nu t}.  The paper prints sin x in w; with cos x the
    field satisfies curl v = v, which is what makes it an exact solution."""
    e = math.exp(-nu * t)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    return ((np.sin(z) + np.cos(y)) * e, (np.sin(x) + np.cos(z)) * e,
            (np.sin(y) + np.cos(x)) * e)


def abc_pressure(x, y, z, t=0.0, nu=0.0):
    """Pressure of the ABC flow: for a Beltrami field the convective term is
    grad(|v|^2 / 2), so p = -|v|^2 / 2."""
    u, v, w = abc_flow(x, y, z, t, nu)
    return -0.5 * (u * u + v * v + w * w)


# ---------------------------------------------------------------- perturbations
@dataclasses.dataclass(frozen=True)
class StreamModes:
    """Stream function psi(x, y) = sum_m a[m] sin(kx[m] x + ky[m] y + phase[m])."""
    kx: np.ndarray
    ky: np.ndarray
    phase: np.ndarray
    a: np.ndarray


def stream_modes(seed: int, nmodes: int, kmax: int, amplitude: float,
                 period: float = 2.0 * math.pi) -> StreamModes:
    """Draw `nmodes` integer wave vectors with 1 <= max(|kx|,|ky|) <= kmax
    (in units of 2 pi / period), uniform phases, and coefficients uniform in
    [-1, 1]; then scale the coefficients so that max |grad psi| over a
    512 x 512 sample grid of the periodic box equals `amplitude`."""
    rng = np.random.default_rng(seed)
    kx = np.empty(nmodes, dtype=np.int64)
    ky = np.empty(nmodes, dtype=np.int64)
    m = 0
    while m < nmodes:
        a, b = rng.integers(-kmax, kmax + 1, size=2)
        if max(abs(a), abs(b)) >= 1:
            kx[m], ky[m] = a, b
            m += 1
    phase = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
    coef = rng.uniform(-1.0, 1.0, size=nmodes)
    k0 = 2.0 * math.pi / period
    modes = StreamModes(kx * k0, ky * k0, phase, coef)
    s = np.linspace(0.0, period, 512, endpoint=False)
    X, Y = np.meshgrid(s, s, indexing="xy")
    u, v = perturbation_velocity(modes, X, Y)
    vmax = float(np.max(np.sqrt(u * u + v * v)))
    scale = amplitude / vmax if vmax > 0 else 0.0
    return StreamModes(modes.kx, modes.ky, phase, coef * scale)


def perturbation_velocity(modes: StreamModes, x, y):
    """Velocity (d psi/dy, -d psi/dx) of the stream function `modes`."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    u = np.zeros(np.broadcast(x, y).shape)
    v = np.zeros_like(u)
    for kx, ky, ph, a in zip(modes.kx, modes.ky, modes.phase, modes.a):
        c = a * np.cos(kx * x + ky * y + ph)
        u += ky * c
        v -= kx * c
    return u, v


# ---------------------------------------------------------------- batches
@dataclasses.dataclass(frozen=True)
class BatchMember:
    cells: int     # cells per side (2D, square periodic box)
    N: int         # polynomial degree
    nu: float      # kinematic viscosity


def batch_members(seed: int, count: int,
                  cells=(16, 32, 64, 128), degrees=(2, 11),
                  nu_range=(1e-4, 1e-1)) -> list[BatchMember]:
    """Independent problems of uneven size: cells per side drawn from `cells`,
    N uniform in the closed range `degrees`, nu log-uniform in `nu_range`."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = math.log(nu_range[0]), math.log(nu_range[1])
    for _ in range(count):
        c = int(rng.choice(np.asarray(cells)))
        n = int(rng.integers(degrees[0], degrees[1] + 1))
        nu = float(math.exp(rng.uniform(lo, hi)))
        out.append(BatchMember(c, n, nu))
    return out


def random_vector(seed: int, n: int) -> np.ndarray:
    """Standard-normal FP64 vector of length n (operator and solver inputs)."""
    return np.random.default_rng(seed).standard_normal(n)
