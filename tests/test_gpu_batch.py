"""Batches of independent problems (sdg_batch_*) on the GPU: every member
matches the same problem stepped alone (bit for bit: same kernels, same
deterministic reductions) and the oracle."""
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

from oracle import Grid, Oracle  # noqa: E402
import sdg_inputs as si  # noqa: E402
from paper_1602_05806_gb300 import sdg  # noqa: E402
from paper_1602_05806_gb300.workloads import batch_workload, taylor_green_state  # noqa: E402

TWO_PI = 2.0 * math.pi


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _state(dim, n, L, N, seed):
    if dim == 2:
        modes = si.stream_modes(seed, 8, 8, 1e-2)
        return taylor_green_state(2, n, L, N, modes=modes), modes
    return taylor_green_state(3, n, L, N), None


def _oracle_state(o, modes):
    U = []
    if o.dim == 2:
        for d in range(2):
            x, y = o.coords(d)
            v = si.taylor_green_2d(x, y)[d]
            if modes is not None:
                v = v + si.perturbation_velocity(modes, x, y)[d]
            U.append(v)
        x, y = o.coords(None)
        P = si.taylor_green_2d(x, y)[2]
    else:
        for d in range(3):
            U.append(si.taylor_green_3d(*o.coords(d))[d])
        P = si.taylor_green_3d(*o.coords(None))[3]
    return U, P


# uneven sizes and degrees, both precisions, 2D and 3D
PROBLEMS = [
    (2, (8, 8), (TWO_PI, TWO_PI), 3, 0.1, sdg.SDG_FP64),
    (2, (6, 10), (TWO_PI, TWO_PI), 5, 0.01, sdg.SDG_MIXED),
    (2, (12, 12), (TWO_PI, TWO_PI), 2, 1e-3, sdg.SDG_MIXED),
    (3, (3, 4, 3), (TWO_PI,) * 3, 2, 0.02, sdg.SDG_FP64),
    (2, (5, 7), (TWO_PI, TWO_PI), 7, 1e-4, sdg.SDG_FP64),
    (2, (4, 6), (TWO_PI, TWO_PI), 11, 0.05, sdg.SDG_MIXED),
]


def test_batch_members_match_single_handles_and_oracle():
    theta, dt, steps = 0.51, 1e-3, 2
    b = sdg.Batch([p[:5] for p in PROBLEMS], theta, dt)
    singles, oracles = [], []
    for i, (dim, n, L, N, nu, prec) in enumerate(PROBLEMS):
        (Ug, Pg), modes = _state(dim, n, L, N, 100 + i)
        for h in (b.members[i], sdg.Handle(dim, n, L, N, nu, theta, dt)):
            h.set_options(prec, 1e-13, 1e-13, 1000000)
            h.set_state([dev(u) for u in Ug], dev(Pg))
            if h is not b.members[i]:
                singles.append(h)
        o = Oracle(Grid(dim, n, L), N, nu, theta, dt, rtol_p=1e-13, rtol_v=1e-13)
        oracles.append((o, *_oracle_state(o, modes)))
    b.set_threads(3)
    rc, infos = b.step(steps)
    assert rc == sdg.SDG_OK and all(inf["status"] == sdg.SDG_OK for inf in infos)
    for i, (dim, n, L, N, nu, prec) in enumerate(PROBLEMS):
        singles[i].step(steps)
        shape = b.members[i].shape
        Ub = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(dim)]
        Us = [torch.empty_like(Ub[0]) for _ in range(dim)]
        Pb, Ps = torch.empty_like(Ub[0]), torch.empty_like(Ub[0])
        b.members[i].get_state(Ub, Pb)
        singles[i].get_state(Us, Ps)
        for d in range(dim):
            assert torch.equal(Ub[d], Us[d]), (i, d)
        assert torch.equal(Pb, Ps), i
        # oracle with both linear systems solved exactly (block-circulant
        # Fourier solve): the comparison then carries only the GPU's CG error
        o, U, P = oracles[i]
        for _ in range(steps):
            U, P = o.step_exact(U, P)
        tol = 1e-11 if prec == sdg.SDG_FP64 else 1e-10
        for d in range(dim):
            assert rel(host(Ub[d]), U[d]) <= tol, (i, d)
        # the mixed solve may stop at its FP64 true-residual floor (up to
        # 10 rtol, relative to a right-hand side that is small against A' P
        # at dt = 1e-3), which the smoothest pressure modes amplify
        assert rel(host(Pb), P) <= (1e-10 if prec == sdg.SDG_FP64 else 1e-8), i
        singles[i].close()
    b.close()


def test_batch_workload_48_problems_one_step():
    """The 48-problem batch (seed 2: 16^2..128^2 cells, N = 2..11, 17.4 M DOF
    per field in total), one mixed-precision step of every member at
    rtol 1e-12: every solve converges, and the two smallest members match
    the oracle."""
    w, problems, states = batch_workload()
    b = sdg.Batch(problems, w["theta"], w["dt"])
    for i, (U, P) in enumerate(states):
        m = b.members[i]
        m.set_options(sdg.SDG_MIXED, 1e-12, 1e-12, 1000000)
        m.set_convection_substeps(w["nsub"][i])
        m.set_state([dev(u) for u in U], dev(P))
    rc, infos = b.step(1)
    assert rc == sdg.SDG_OK
    for i, inf in enumerate(infos):
        assert inf["status"] == sdg.SDG_OK and inf["pressure"]["rel_res"] <= 1e-11, (i, inf)
    sizes = [p[1][0] * p[1][1] * (p[3] + 1) ** 2 for p in problems]
    for i in sorted(range(len(problems)), key=lambda k: sizes[k])[:2]:
        dim, n, L, N, nu = problems[i]
        o = Oracle(Grid(dim, n, L), N, nu, w["theta"], w["dt"], rtol_p=1e-13, rtol_v=1e-13)
        modes = si.stream_modes(1000 * w["seed"] + i, w["nmodes"], w["kmax"], w["amplitude"])
        U, P = _oracle_state(o, modes)
        U, P = o.step_exact(U, P)
        shape = b.members[i].shape
        Ub = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(dim)]
        Pb = torch.empty_like(Ub[0])
        b.members[i].get_state(Ub, Pb)
        for d in range(dim):
            assert rel(host(Ub[d]), U[d]) <= 1e-10, (i, d)
        assert rel(host(Pb), P) <= 1e-9, i
    b.close()
