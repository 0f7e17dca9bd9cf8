"""Pins of the oracle's tangent (JVP) and adjoint (VJP) of one time step
against what fixes them independently: central finite differences of the
forward step (Oracle.step_exact), and the dot-product identity
<VJP(lam), v> = <lam, JVP(v)> that defines the transpose."""
import math

import numpy as np
import pytest

from oracle import Adjoint, Grid, Oracle
import sdg_inputs as si

TWO_PI = 2.0 * math.pi


def _state(o, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    if o.dim == 2:
        modes = si.stream_modes(seed, 6, 3, amp)
        U = []
        for d in range(2):
            x, y = o.coords(d)
            U.append(si.taylor_green_2d(x, y)[d] + si.perturbation_velocity(modes, x, y)[d])
        x, y = o.coords(None)
        P = si.taylor_green_2d(x, y)[2]
    else:
        U = [si.taylor_green_3d(*o.coords(d))[d] + amp * rng.standard_normal(o.shape) for d in range(3)]
        P = si.taylor_green_3d(*o.coords(None))[3]
    return U, P - o.physical_mean(P)


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


CASES = [(2, (5, 4), 3, 1), (2, (4, 4), 2, 2), (3, (3, 2, 2), 2, 1)]


@pytest.mark.parametrize("dim,n,N,nsub", CASES)
def test_convection_tangent_matches_finite_differences(dim, n, N, nsub):
    o = Oracle(Grid(dim, n, (TWO_PI,) * dim), N, 0.02, 0.55, 0.05, nsub=nsub)
    A = Adjoint(o)
    V, _ = _state(o, 3)
    rng = np.random.default_rng(4)
    dV = [rng.standard_normal(o.shape) for _ in range(dim)]
    eps = 1e-6
    Lp = o.convection([v + eps * e for v, e in zip(V, dV)])
    Lm = o.convection([v - eps * e for v, e in zip(V, dV)])
    J = A.convection_jvp(V, dV)
    for c in range(dim):
        fd = (Lp[c] - Lm[c]) / (2 * eps)
        assert np.linalg.norm(J[c] - fd) <= 1e-7 * np.linalg.norm(fd), c


@pytest.mark.parametrize("dim,n,N,nsub", CASES)
def test_convection_and_rk3_adjoint_dot_products(dim, n, N, nsub):
    o = Oracle(Grid(dim, n, (TWO_PI,) * dim), N, 0.02, 0.55, 0.05, nsub=nsub)
    A = Adjoint(o)
    V, _ = _state(o, 5)
    rng = np.random.default_rng(6)
    v = [rng.standard_normal(o.shape) for _ in range(dim)]
    lam = [rng.standard_normal(o.shape) for _ in range(dim)]
    lhs, rhs = _dot(A.convection_vjp(V, lam), v), _dot(lam, A.convection_jvp(V, v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    lhs, rhs = _dot(A.rk3_vjp(V, lam), v), _dot(lam, A.rk3_jvp(V, v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("dim,n,N,nsub", CASES)
def test_step_tangent_matches_finite_differences(dim, n, N, nsub):
    """Directional derivative of step_exact in (U, P, nu) by central
    differences (eps 1e-6) against step_jvp."""
    o = Oracle(Grid(dim, n, (TWO_PI,) * dim), N, 0.02, 0.55, 0.05, nsub=nsub)
    A = Adjoint(o)
    U, P = _state(o, 7)
    rng = np.random.default_rng(8)
    dU = [rng.standard_normal(o.shape) for _ in range(dim)]
    dP = rng.standard_normal(o.shape)
    dnu = 0.7
    eps = 1e-6

    def run(s):
        o.nu = 0.02 + s * eps * dnu
        Un, Pn = o.step_exact([u + s * eps * e for u, e in zip(U, dU)], P + s * eps * dP)
        o.nu = 0.02
        return Un, Pn

    Up, Pp = run(+1)
    Um, Pm = run(-1)
    JU, JP = A.step_jvp(U, P, dU, dP, dnu)
    for d in range(dim):
        fd = (Up[d] - Um[d]) / (2 * eps)
        assert np.linalg.norm(JU[d] - fd) <= 1e-7 * np.linalg.norm(fd), d
    fd = (Pp - Pm) / (2 * eps)
    assert np.linalg.norm(JP - fd) <= 1e-7 * np.linalg.norm(fd)


@pytest.mark.parametrize("dim,n,N,nsub", CASES)
def test_step_adjoint_dot_product(dim, n, N, nsub):
    """<step_vjp(lam), (v, dnu)> = <lam, step_jvp(v, dnu)> in (U, P, nu)."""
    o = Oracle(Grid(dim, n, (TWO_PI,) * dim), N, 0.02, 0.55, 0.05, nsub=nsub)
    A = Adjoint(o)
    U, P = _state(o, 9)
    rng = np.random.default_rng(10)
    vU = [rng.standard_normal(o.shape) for _ in range(dim)]
    vP = rng.standard_normal(o.shape)
    vnu = 0.3
    lU = [rng.standard_normal(o.shape) for _ in range(dim)]
    lP = rng.standard_normal(o.shape)
    JU, JP = A.step_jvp(U, P, vU, vP, vnu)
    gU, gP, gnu = A.step_vjp(U, P, lU, lP)
    lhs = _dot(gU, vU) + float(np.sum(gP * vP)) + gnu * vnu
    rhs = _dot(lU, JU) + float(np.sum(lP * JP))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_loss_gradient_over_steps_matches_finite_differences():
    """Loss 0.5 ||u(T) - u_TG(T)||^2 after three steps: the adjoint sweep
    (step_vjp backwards through the saved states) gives d loss / d U0 along
    a random direction and d loss / d nu that agree with central
    differences."""
    o = Oracle(Grid(2, (4, 4), (TWO_PI, TWO_PI)), 3, 0.05, 0.51, 0.02)
    A = Adjoint(o)
    U0, P0 = _state(o, 11)
    T = 3 * o.dt
    target = []
    for d in range(2):
        x, y = o.coords(d)
        target.append(si.taylor_green_2d(x, y, T, o.nu)[d])

    def loss(U, P, nu):
        o.nu = nu
        for _ in range(3):
            U, P = o.step_exact(U, P)
        o.nu = 0.05
        return 0.5 * sum(float(np.sum((U[d] - target[d]) ** 2)) for d in range(2))

    states = [(U0, P0)]
    U, P = U0, P0
    for _ in range(3):
        U, P = o.step_exact(U, P)
        states.append((U, P))
    lU = [U[d] - target[d] for d in range(2)]
    lP = np.zeros(o.shape)
    gnu = 0.0
    for k in reversed(range(3)):
        lU, lP, g = A.step_vjp(states[k][0], states[k][1], lU, lP)
        gnu += g
    rng = np.random.default_rng(12)
    v = [rng.standard_normal(o.shape) for _ in range(2)]
    eps = 1e-6
    fd = (loss([u + eps * e for u, e in zip(U0, v)], P0, 0.05)
          - loss([u - eps * e for u, e in zip(U0, v)], P0, 0.05)) / (2 * eps)
    assert abs(_dot(lU, v) - fd) <= 1e-6 * abs(fd)
    fd_nu = (loss(U0, P0, 0.05 + eps) - loss(U0, P0, 0.05 - eps)) / (2 * eps)
    assert abs(gnu - fd_nu) <= 1e-6 * abs(fd_nu)
