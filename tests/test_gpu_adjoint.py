"""The library's adjoint of the time step (sdg_step_adjoint) on the GPU:
against the oracle's adjoint on small grids, and the gradient of a loss over
20 steps of the 64 x 64, N = 5 workload against central finite differences
of the GPU's own forward steps."""
import math
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")

from oracle import Adjoint, Grid, Oracle  # noqa: E402
import sdg_inputs as si  # noqa: E402
from paper_1602_05806_gb300 import sdg  # noqa: E402
from paper_1602_05806_gb300.autograd import steps  # noqa: E402
from paper_1602_05806_gb300.workloads import taylor_green_state, workload_state, coords  # noqa: E402

TWO_PI = 2.0 * math.pi


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,N,nsub,prec", [(2, (5, 4), 3, 1, sdg.SDG_FP64), (2, (4, 4), 2, 2, sdg.SDG_FP64),
                                               (3, (3, 2, 2), 2, 1, sdg.SDG_FP64), (2, (6, 5), 5, 1, sdg.SDG_MIXED)])
def test_step_adjoint_matches_oracle(dim, n, N, nsub, prec):
    L = (TWO_PI,) * dim
    nu, theta, dt = 0.02, 0.55, 0.05
    o = Oracle(Grid(dim, n, L), N, nu, theta, dt, nsub=nsub)
    A = Adjoint(o)
    rng = np.random.default_rng(21)
    if dim == 2:
        U, P = taylor_green_state(2, n, L, N, modes=si.stream_modes(5, 6, 3, 0.05))
    else:
        U, P = taylor_green_state(3, n, L, N)
        U = [u + 0.05 * rng.standard_normal(u.shape) for u in U]
    lU = [rng.standard_normal(o.shape) for _ in range(dim)]
    lP = rng.standard_normal(o.shape)
    gU, gP, gnu = A.step_vjp(U, P, lU, lP)
    h = sdg.Handle(dim, n, L, N, nu, theta, dt)
    h.set_convection_substeps(nsub)
    h.set_options(prec, 1e-14 if prec == sdg.SDG_FP64 else 1e-13, 1e-14 if prec == sdg.SDG_FP64 else 1e-13)
    LU = [dev(x) for x in lU]
    LP = dev(lP)
    dnu = h.step_adjoint([dev(u) for u in U], LU, LP)
    tol = 1e-9 if prec == sdg.SDG_FP64 else 1e-8
    for d in range(dim):
        assert rel(host(LU[d]), gU[d]) <= tol, d
    assert rel(host(LP), gP) <= tol
    assert abs(dnu - gnu) <= tol * abs(gnu)
    h.close()


def _tg_target(n, L, N, T, nu):
    out = []
    for d in range(2):
        x, y = coords(2, n, L, N, d)
        out.append(si.taylor_green_2d(x, y, T, nu)[d])
    return out


def test_loss_gradient_64x64_N5_against_finite_differences():
    """Loss 0.5 ||u(T) - u_TG(T)||^2 after 20 steps of the 64 x 64, N = 5
    workload (TG + 16 modes, seed 1, amplitude 0.05, nu 0.01, dt 5e-3, three
    convection sub-steps).  d loss / d U0 along 16 seeded random directions
    and d loss / d nu from the adjoint agree with central differences
    (eps 1e-6) of the forward steps within 1e-6 (relative to the gradient
    norm for the unit directions)."""
    w, U0, P0 = workload_state("tg2d_64x64_N5")
    nsteps = w["steps"]
    T = nsteps * w["dt"]
    target = [dev(t) for t in _tg_target(w["n"], w["L"], w["N"], T, w["nu"])]

    def handle(nu):
        h = sdg.Handle(2, w["n"], w["L"], w["N"], nu, w["theta"], w["dt"])
        h.set_convection_substeps(w["nsub"])
        # rtol 1e-13: tight enough that the solver noise over eps stays far
        # below the 1e-6 target; plain FP64 CG on this singular system breaks
        # down (p^T A p <= 0) when asked for 1e-14, below its round-off floor
        h.set_options(sdg.SDG_FP64, 1e-13, 1e-13)
        return h

    def loss_of(h, U, P, nu):
        UT, _ = steps(h, U, P, nu, nsteps)
        return 0.5 * sum(((UT[d] - target[d]) ** 2).sum() for d in range(2))

    h = handle(w["nu"])
    U = [dev(u).requires_grad_(True) for u in U0]
    P = dev(P0)
    nu = torch.tensor(w["nu"], dtype=torch.float64, requires_grad=True)
    loss = loss_of(h, U, P, nu)
    loss.backward()
    g = [u.grad.detach() for u in U]
    gnorm = math.sqrt(sum(float((x * x).sum()) for x in g))
    gnu = float(nu.grad)
    eps = 1e-6
    rng = np.random.default_rng(1)
    with torch.no_grad():
        for k in range(16):
            v = [dev(rng.standard_normal(U0[0].shape)) for _ in range(2)]
            s = 1.0 / math.sqrt(sum(float((x * x).sum()) for x in v))
            v = [x * s for x in v]
            lp = float(loss_of(h, [u.detach() + eps * x for u, x in zip(U, v)], P, nu.detach()))
            lm = float(loss_of(h, [u.detach() - eps * x for u, x in zip(U, v)], P, nu.detach()))
            fd = (lp - lm) / (2 * eps)
            ad = sum(float((gi * x).sum()) for gi, x in zip(g, v))
            # unit directions: the scale of a directional derivative is the
            # gradient norm (|fd| itself can be far smaller for a random
            # direction, and then carries the round-off of the loss / eps)
            assert abs(ad - fd) <= 1e-6 * max(abs(fd), gnorm), (k, ad, fd, gnorm)
        hp, hm = handle(w["nu"] + eps), handle(w["nu"] - eps)
        lp = float(loss_of(hp, [u.detach() for u in U], P, torch.tensor(w["nu"] + eps, dtype=torch.float64)))
        lm = float(loss_of(hm, [u.detach() for u in U], P, torch.tensor(w["nu"] - eps, dtype=torch.float64)))
        fd = (lp - lm) / (2 * eps)
        assert abs(gnu - fd) <= 1e-6 * abs(fd), (gnu, fd)
    for x in (h, hp, hm):
        x.close()
