"""Pins of the CPU oracle against facts the paper and the mathematics fix
(no GPU).  Each test names the passage it checks.  A plausible slip in the
oracle (a dropped jump term, a wrong sign, a transposed matrix, a wrong roll
direction) fails at least one of them."""
import math
import os

import numpy as np
import pytest

from oracle import Basis, Grid, Oracle, cg, gauss_legendre_01, lagrange, lagrange_deriv
import sdg_inputs as si

TWO_PI = 2.0 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def J(n1):
    return np.fliplr(np.eye(n1))


# ------------------------------------------------------------------ Sec. 2.1 basis
@pytest.mark.parametrize("N", range(0, 12))
def test_gauss_legendre_exactness(N):
    """GL rule with n1 = N+1 points integrates monomials of degree <= 2N+1
    exactly and is symmetric about 1/2 (basis of Sec. 2.1)."""
    xi, w = gauss_legendre_01(N + 1)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * N + 2):
        assert abs(np.sum(w * xi**k) - 1.0 / (k + 1)) < 1e-14
    if 1 <= N <= 6:  # degree 2N+2 is not exact (its error shrinks fast with N)
        k = 2 * N + 2
        assert abs(np.sum(w * xi**k) - 1.0 / (k + 1)) > 1e-12
    assert np.allclose(xi + xi[::-1], 1.0, atol=1e-15)
    assert np.allclose(w, w[::-1], atol=1e-15)


@pytest.mark.parametrize("N", [1, 3, 7, 11])
def test_lagrange_basis(N):
    xi, _ = gauss_legendre_01(N + 1)
    V = np.array([[lagrange(xi, p, xi[q]) for q in range(N + 1)] for p in range(N + 1)])
    assert np.allclose(V, np.eye(N + 1), atol=1e-13)
    s = np.linspace(0, 1, 17)
    assert np.allclose(sum(lagrange(xi, p, s) for p in range(N + 1)), 1.0, atol=1e-11)
    assert np.allclose(sum(lagrange_deriv(xi, p, s) for p in range(N + 1)), 0.0, atol=1e-8)
    h = 1e-6
    for p in range(N + 1):
        fd = (lagrange(xi, p, s + h) - lagrange(xi, p, s - h)) / (2 * h)
        assert np.allclose(lagrange_deriv(xi, p, s), fd, rtol=1e-6, atol=1e-5 * max(1, N**2))


@pytest.mark.parametrize("N", range(0, 12))
def test_mass_matrix_diagonal(N):
    """Sec. 2.1: the nodal GL basis is orthogonal, M = diag(w)."""
    B = Basis(N)
    assert np.allclose(B.M, np.diag(B.w), atol=1e-14)


def test_N0_matrices():
    """N = 0 (Sec. 3.3, last paragraph: M = N = 0 gives the classical
    staggered scheme): every 1D matrix is 1 and H = (-1, 2, -1)."""
    B = Basis(0)
    for m in (B.M, B.Rt, B.Lt, B.Rb, B.Lb):
        assert np.allclose(m, 1.0)
    assert np.allclose(B.HR, -1.0) and np.allclose(B.HL, -1.0) and np.allclose(B.HC, 2.0)
    assert np.allclose(B.ML, 0.5) and np.allclose(B.MR, 0.5)


# ------------------------------------------------------------------ Eq. matrices
@pytest.mark.parametrize("N", range(0, 12))
def test_transpose_identities(N):
    """Eq. matricesLR: R~ = L-bar^T and L~ = R-bar^T (each side computed from
    its own integral); M^R = (M^L)^T (Sec. 2.2)."""
    B = Basis(N)
    assert np.allclose(B.Rt, B.Lb.T, atol=1e-13)
    assert np.allclose(B.Lt, B.Rb.T, atol=1e-13)
    assert np.allclose(B.MR, B.ML.T, atol=1e-14)


@pytest.mark.parametrize("N", range(1, 12))
def test_reflection_symmetry(N):
    """Derived: mirroring xi -> 1 - xi maps the right half-cell onto the left,
    so L~ = J R~ J, H^L = J H^R J and J H^C J = H^C."""
    B = Basis(N)
    j = J(N + 1)
    assert np.allclose(B.Lt, j @ B.Rt @ j, atol=1e-12)
    scale = np.abs(B.HC).max()
    assert np.allclose(B.HL, j @ B.HR @ j, atol=1e-13 * scale)
    assert np.allclose(B.HC, j @ B.HC @ j, atol=1e-13 * scale)


@pytest.mark.parametrize("N", range(0, 12))
def test_gradient_of_constant(N):
    """R~ 1 = L~ 1 = phi(1/2): the weak gradient of a constant vanishes and a
    unit jump contributes exactly phi_p(1/2) (Eq. pressurejump)."""
    B = Basis(N)
    half = np.array([lagrange(B.xi, p, 0.5) for p in range(N + 1)])
    one = np.ones(N + 1)
    assert np.allclose(B.Rt @ one, half, atol=1e-13)
    assert np.allclose(B.Lt @ one, half, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 12))
def test_weak_gradient_reproduces_polynomials(N):
    """Eq. uDGNSmom / pressurejump in reference units (dx = 1): for a single
    polynomial p of degree <= N spanning main cells i (x in [0,1]) and i+1
    (x in [1,2]), the dual cell i+1/2 = [1/2, 3/2] gives
        R~ P_{i+1} - L~ P_i = w_m p'(1/2 + xi_m)      (exact GL quadrature),
    and adding a jump c to cell i+1 adds c phi_m(1/2)."""
    B = Basis(N)
    rng = np.random.default_rng(N)
    c = rng.standard_normal(N + 1)
    p = np.polynomial.Polynomial(c)
    Pi, Pi1 = p(B.xi), p(1.0 + B.xi)
    lhs = B.Rt @ Pi1 - B.Lt @ Pi
    rhs = B.w * p.deriv()(0.5 + B.xi)
    assert np.allclose(lhs, rhs, atol=1e-11 * max(1.0, np.abs(rhs).max()))
    jump = 0.7
    half = np.array([lagrange(B.xi, m, 0.5) for m in range(N + 1)])
    assert np.allclose(B.Rt @ (Pi1 + jump) - B.Lt @ Pi, rhs + jump * half, atol=1e-10)


@pytest.mark.parametrize("N", range(1, 12))
def test_weak_divergence_reproduces_polynomials(N):
    """Eq. DGNSinc2 in reference units: main cell i = [0,1], dual cells
    i-1/2 = [-1/2, 1/2] and i+1/2 = [1/2, 3/2]; for one polynomial u of degree
    <= N,  R-bar U_{i+1/2} - L-bar U_{i-1/2} = w_m u'(xi_m)."""
    B = Basis(N)
    rng = np.random.default_rng(100 + N)
    u = np.polynomial.Polynomial(rng.standard_normal(N + 1))
    Um, Up = u(-0.5 + B.xi), u(0.5 + B.xi)
    lhs = B.Rb @ Up - B.Lb @ Um
    rhs = B.w * u.deriv()(B.xi)
    assert np.allclose(lhs, rhs, atol=1e-11 * max(1.0, np.abs(rhs).max()))


@pytest.mark.parametrize("N", range(0, 12))
def test_projection_reproduces_polynomials(N):
    """Eqs. l2forward / l2backward: the L2 projection between half-overlapping
    cells is exact for one polynomial of degree <= N."""
    B = Basis(N)
    rng = np.random.default_rng(200 + N)
    u = np.polynomial.Polynomial(rng.standard_normal(N + 1))
    # dual -> main: main cell [0,1], duals [-1/2,1/2] and [1/2,3/2]
    main = B.Minv @ (B.ML @ u(-0.5 + B.xi) + B.MR @ u(0.5 + B.xi))
    assert np.allclose(main, u(B.xi), atol=1e-12 * max(1, np.abs(u(B.xi)).max()))
    # main -> dual: dual [1/2,3/2] from mains [0,1] and [1,2]
    dual = B.Minv @ (B.ML @ u(B.xi) + B.MR @ u(1.0 + B.xi))
    assert np.allclose(dual, u(0.5 + B.xi), atol=1e-12 * max(1, np.abs(dual).max()))


@pytest.mark.parametrize("N", range(0, 12))
def test_H_blocks_symmetry(N):
    """Sec. 2.1 symmetry proof: (H^R)^T = H^L and (H^C)^T = H^C."""
    B = Basis(N)
    s = max(1.0, np.abs(B.HC).max())
    assert np.allclose(B.HR.T, B.HL, atol=1e-13 * s)
    assert np.allclose(B.HC.T, B.HC, atol=1e-13 * s)


# ------------------------------------------------------------------ Eq. pSyst, dense
def _oracle(dim, n, N, L=None, nu=0.05, theta=0.6, dt=0.03):
    L = L or tuple([TWO_PI] * dim)
    return Oracle(Grid(dim, n, L), N, nu, theta, dt)


def test_N0_is_five_point_laplacian():
    """M = N = 0 reduces to the classical staggered finite-difference scheme:
    theta A' is theta dt times the periodic 5-point Laplacian, whose
    eigenvalues are theta dt sum_d 4 sin^2(pi k_d / n_d) / dx_d^2."""
    o = _oracle(2, (5, 4), 0, L=(1.0, 2.0))
    A = o.dense(o.pressure_apply)
    ev = np.sort(np.linalg.eigvalsh(A))
    dx, dy = o.g.dx
    ref = sorted(o.theta * o.dt * (4 * math.sin(math.pi * kx / 5) ** 2 / dx**2
                                   + 4 * math.sin(math.pi * ky / 4) ** 2 / dy**2)
                 for kx in range(5) for ky in range(4))
    assert np.allclose(ev, ref, atol=1e-12 * max(ref))


def test_N0_is_seven_point_laplacian_3d():
    o = _oracle(3, (3, 4, 3), 0, L=(1.0, 1.5, 2.0))
    A = o.dense(o.pressure_apply)
    ev = np.sort(np.linalg.eigvalsh(A))
    dx, dy, dz = o.g.dx
    ref = sorted(o.theta * o.dt * (4 * math.sin(math.pi * a / 3) ** 2 / dx**2
                                   + 4 * math.sin(math.pi * b / 4) ** 2 / dy**2
                                   + 4 * math.sin(math.pi * c / 3) ** 2 / dz**2)
                 for a in range(3) for b in range(4) for c in range(3))
    assert np.allclose(ev, ref, atol=1e-12 * max(ref))


def _stencil_golden():
    out = {}
    with open(os.path.join(GOLDEN, "stencil_size.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, b = line.split()
                out[int(d)] = int(b)
    return out


@pytest.mark.parametrize("dim,n,N", [(2, (3, 4), 2), (2, (4, 3), 3), (3, (3, 3, 3), 1),
                                     (3, (3, 3, 3), 2)])
def test_pressure_operator_structure(dim, n, N):
    """Sec. 2.1: H is symmetric, positive semi-definite, and (periodic case)
    its kernel is exactly the set of weak solutions of grad p = 0, i.e. the
    common kernel of the weak gradients D_d.  For even N that is the
    constants alone; for odd N each direction adds one more weak solution
    (a per-cell sawtooth), so the kernel has dimension 2^dim.  Each block row
    has 5 (2D) / 7 (3D) nonzero blocks (Table StencilSize)."""
    o = _oracle(dim, n, N)
    A = o.dense(o.pressure_apply)
    s = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-13 * s
    ev = np.linalg.eigvalsh(A)
    small = np.abs(ev) < 1e-11 * ev.max()
    assert ev[~small].min() > 0
    Dst = np.vstack([o.dense(lambda X: o.weak_gradient(X, d)) for d in range(dim)])
    sv = np.linalg.svd(Dst, compute_uv=False)
    kerD = int(np.sum(sv < 1e-11 * sv.max())) + (Dst.shape[1] - len(sv))
    assert small.sum() == kerD
    assert small.sum() == (1 if N % 2 == 0 else 2 ** dim)
    one = np.ones(A.shape[0])
    assert np.abs(A @ one).max() <= 1e-12 * s
    # block bandwidth
    npe = (N + 1) ** dim
    nb = A.shape[0] // npe
    blocks = np.array([[np.abs(A[i * npe:(i + 1) * npe, j * npe:(j + 1) * npe]).max() > 1e-14 * s
                        for j in range(nb)] for i in range(nb)])
    assert (blocks.sum(axis=1) == _stencil_golden()[dim]).all()


def test_sawtooth_is_weak_constant_N1():
    """N = 1: p = x/dx - i - 1/2 on cell i (slope 1, unit downward jump at each
    face) has zero weak gradient: int psi_m dp = w_m - phi_m(1/2) = 0."""
    o = _oracle(2, (4, 3), 1)
    X, _ = o.coords(None)
    i = np.floor(X / o.g.dx[0] + 1e-12)
    saw = X / o.g.dx[0] - i - 0.5
    assert np.abs(o.weak_gradient(saw, 0)).max() < 1e-13
    assert np.abs(o.pressure_apply(saw)).max() < 1e-13 * np.abs(o.dense(o.pressure_apply)).max()


@pytest.mark.parametrize("dim,n,N", [(2, (3, 4), 2), (3, (3, 2, 3), 2)])
def test_pressure_operator_factorisation(dim, n, N):
    """Eqs. PerPrSyst / weakgradientop: A' = dt sum_d (1/dx_d^2) M^{perp d}
    D_d^T M_d^{-1} D_d with D the weak gradient, and the weak divergence of
    Eq. pSDG1 is -D^T."""
    o = _oracle(dim, n, N)
    A = o.dense(o.Aprime)
    tot = np.zeros_like(A)
    for d in range(dim):
        D = o.dense(lambda X: o.weak_gradient(X, d))
        Dv = o.dense(lambda X: o.weak_divergence(X, d))
        assert np.allclose(Dv, -D.T, atol=1e-12)
        Minv_d = o.dense(lambda X: o.along(o.B.Minv, X, d))
        Mp = o.dense(lambda X: o.mass_perp(X, d))
        tot += (o.dt / o.g.dx[d] ** 2) * Mp @ D.T @ Minv_d @ D
    assert np.allclose(A, tot, atol=1e-12 * np.abs(A).max())


def test_pressure_operator_fourier_symbol():
    """Derived: on a periodic grid the operator is block-circulant; its
    spectrum is the union over wavenumbers of the spectra of the Hermitian
    n1^2 x n1^2 symbols theta dt [ W (x) S_x(kx)/dx^2 + S_y(ky) (x) W / dy^2 ],
    S(k) = H^L e^{-ik} + H^C + H^R e^{ik}."""
    nx, ny, N = 4, 6, 2
    o = _oracle(2, (nx, ny), N, L=(1.0, 1.7))
    A = o.dense(o.pressure_apply)
    ev = np.sort(np.linalg.eigvalsh(A))
    B = o.B
    W = np.diag(B.w)
    ref = []
    for kx in range(nx):
        for ky in range(ny):
            ax, ay = 2 * math.pi * kx / nx, 2 * math.pi * ky / ny
            Sx = B.HL * np.exp(-1j * ax) + B.HC + B.HR * np.exp(1j * ax)
            Sy = B.HL * np.exp(-1j * ay) + B.HC + B.HR * np.exp(1j * ay)
            # local index order (l2, l1): kron(outer=l2, inner=l1)
            S = (np.kron(W, Sx) / o.g.dx[0] ** 2 + np.kron(Sy, W) / o.g.dx[1] ** 2)
            ref.extend(np.linalg.eigvalsh(o.theta * o.dt * S))
    ref = np.sort(ref)
    assert np.allclose(ev, ref, atol=1e-11 * ref.max())


@pytest.mark.parametrize("dim,n,N", [(2, (3, 3), 3), (3, (2, 3, 2), 2)])
def test_viscous_operator_spd(dim, n, N):
    """Eq. implicitviscosity: M + nu H is symmetric positive definite, and
    with nu = 0 it is the diagonal mass matrix."""
    o = _oracle(dim, n, N, nu=0.3)
    A = o.dense(o.viscous_apply)
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= (o.B.w.min() ** dim) * (1 - 1e-12)
    o0 = _oracle(dim, n, N, nu=0.0)
    M = o0.dense(o0.viscous_apply)
    assert np.allclose(M, np.diag(np.diag(M)), atol=1e-15)
    X = np.random.default_rng(3).standard_normal(o0.shape)
    res = cg(o0.viscous_apply, o0.mass_all(X), np.zeros(o0.shape), 1e-14)
    assert np.allclose(res.x, X, atol=1e-13)


# ------------------------------------------------------------------ CG
@pytest.mark.parametrize("dim,n,N", [(2, (4, 3), 3), (2, (3, 4), 2), (3, (2, 2, 3), 2)])
def test_cg_matches_dense_solve(dim, n, N):
    """CG on the singular SPD pressure system, for a compatible b (orthogonal
    to the kernel), equals the kernel part of x0 plus the pseudo-inverse
    solution computed by a dense eigendecomposition."""
    o = _oracle(dim, n, N)
    A = o.dense(o.pressure_apply)
    nd = A.shape[0]
    ev, V = np.linalg.eigh(A)
    ker = np.abs(ev) < 1e-11 * ev.max()
    K = V[:, ker]
    rng = np.random.default_rng(7)
    b = rng.standard_normal(nd)
    b -= K @ (K.T @ b)
    x0 = rng.standard_normal(nd)
    res = cg(lambda X: o.pressure_apply(X), b.reshape(o.shape), x0.reshape(o.shape), 1e-14)
    assert res.converged
    inv = np.where(ker, 0.0, 1.0 / np.where(ker, 1.0, ev))
    xs = K @ (K.T @ x0) + V @ (inv * (V.T @ b))
    assert np.linalg.norm(res.x.ravel() - xs) <= 1e-10 * np.linalg.norm(xs)


def test_cg_zero_rhs_and_breakdown():
    o = _oracle(2, (3, 3), 1)
    x0 = np.ones(o.shape)
    res = cg(o.pressure_apply, np.zeros(o.shape), x0, 1e-12)
    assert res.iters == 0 and np.array_equal(res.x, x0)


# ------------------------------------------------------------------ Sec. 2.2 convection
def test_convection_free_stream():
    """A constant velocity field is an exact steady state of the explicit
    convective operator (Eqs. Fu-Fw, Rusanov flux)."""
    o = _oracle(2, (4, 5), 3)
    V = [np.full(o.shape, 0.7), np.full(o.shape, -0.3)]
    Lv = o.convection(V)
    assert max(np.abs(x).max() for x in Lv) < 1e-12
    o3 = _oracle(3, (3, 3, 2), 2)
    V = [np.full(o3.shape, 0.2), np.full(o3.shape, -0.4), np.full(o3.shape, 1.1)]
    assert max(np.abs(x).max() for x in o3.convection(V)) < 1e-12


def test_convection_conservation():
    """Periodic DG with a single-valued numerical flux conserves each momentum
    component: sum over cells of int L(V)_c dx = 0."""
    o = _oracle(2, (5, 4), 3)
    rng = np.random.default_rng(11)
    V = [rng.standard_normal(o.shape) for _ in range(2)]
    for Lc in o.convection(V):
        assert abs(np.sum(o.mass_all(Lc))) < 1e-11 * np.abs(Lc).max()


@pytest.mark.parametrize("N", [2, 3])
def test_convection_accuracy_order(N):
    """For the Taylor-Green field, div(v v) = (sin 2x / 2, sin 2y / 2); the DG
    operator approaches -div(v v) at order >= N under refinement."""
    errs = []
    for n in (8, 16, 32):
        o = _oracle(2, (n, n), N)
        X, Y = o.coords(None)
        u, v, _ = si.taylor_green_2d(X, Y)
        Lv = o.convection([u, v])
        errs.append(max(np.abs(Lv[0] + 0.5 * np.sin(2 * X)).max(),
                        np.abs(Lv[1] + 0.5 * np.sin(2 * Y)).max()))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= N - 0.2, orders


def test_rk3_coefficients(monkeypatch):
    """SSP-RK3 (reading R9) applied to dV/dt = lambda V gives the cubic Taylor
    polynomial 1 + z + z^2/2 + z^3/6, z = lambda dt."""
    o = _oracle(2, (2, 2), 1, dt=0.3)
    lam = -1.7
    monkeypatch.setattr(o, "convection", lambda V: [lam * x for x in V])
    V = [np.ones(o.shape), 2 * np.ones(o.shape)]
    out = o.rk3(V)
    z = lam * o.dt
    g = 1 + z + z * z / 2 + z**3 / 6
    assert np.allclose(out[0], g) and np.allclose(out[1], 2 * g)


@pytest.mark.parametrize("nsub", [2, 5])
def test_rk3_substeps(monkeypatch, nsub):
    """Reading R12: nsub sub-steps of length dt / nsub.  On dV/dt = lambda V
    the result is the cubic Taylor factor of z / nsub raised to nsub."""
    o = _oracle(2, (2, 2), 1, dt=0.9)
    o.nsub = nsub
    lam = -2.3
    monkeypatch.setattr(o, "convection", lambda V: [lam * x for x in V])
    V = [np.ones(o.shape), -np.ones(o.shape)]
    out = o.rk3(V)
    z = lam * o.dt / nsub
    g = (1 + z + z * z / 2 + z**3 / 6) ** nsub
    assert np.allclose(out[0], g, rtol=1e-14) and np.allclose(out[1], -g, rtol=1e-14)


def test_subcycling_above_cfl_limit():
    """Eq. CFL1 bounds the explicit convection to CFL < 1.  The perturbed
    Taylor-Green field at CFL 2.44 (8x8 cells, N=7, dt=0.064) blows up within
    a few steps with one RK3 step per dt, and decays smoothly with five
    sub-steps of CFL 0.49 each (reading R12)."""
    n, N, dt = 8, 7, 0.064
    cfl = dt * (2 * N + 1) * 2 * n / TWO_PI
    assert 2.4 < cfl < 2.5
    modes = si.stream_modes(0, 32, 8, 1e-2)
    ke = {}
    for nsub in (1, 5):
        o = Oracle(Grid(2, (n, n), (TWO_PI, TWO_PI)), N, 1e-3, 0.51, dt, rtol_p=1e-10, rtol_v=1e-10,
                   nsub=nsub)
        U = []
        for d in range(2):
            x, y = o.coords(d)
            U.append(si.taylor_green_2d(x, y)[d] + si.perturbation_velocity(modes, x, y)[d])
        x, y = o.coords(None)
        P = si.taylor_green_2d(x, y)[2]
        ke[nsub] = [o.kinetic_energy(U)]
        with np.errstate(all="ignore"):
            for _ in range(6):
                U, P, _ = o.step(U, P)
                ke[nsub].append(o.kinetic_energy(U))
    assert not (ke[1][-1] < 10 * ke[1][0]), ke[1]          # unstable (or NaN)
    k5 = np.array(ke[5])
    assert np.all(np.diff(k5) < 0) and k5[-1] > 0.98 * k5[0], k5


def test_projection_accuracy_order():
    """Eq. l2forward on a smooth field: the projection from the dual to the main
    grid converges at order N+1 in the max norm."""
    N = 3
    errs = []
    for n in (8, 16, 32):
        o = _oracle(2, (n, n), N)
        Xu, Yu = o.coords(0)
        X, Y = o.coords(None)
        u = si.taylor_green_2d(Xu, Yu)[0]
        um = o.dual_to_main(u, 0)
        errs.append(np.abs(um - si.taylor_green_2d(X, Y)[0]).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= N + 1 - 0.3, orders


# ------------------------------------------------------------------ Sec. 2.3 step
def _tg_state(o, t=0.0):
    Xu, Yu = o.coords(0)
    Xv, Yv = o.coords(1)
    X, Y = o.coords(None)
    u = si.taylor_green_2d(Xu, Yu, t, o.nu)[0]
    v = si.taylor_green_2d(Xv, Yv, t, o.nu)[1]
    p = si.taylor_green_2d(X, Y, t, o.nu)[2]
    return [u, v], p - o.physical_mean(p)


def test_step_divergence_free():
    """Eq. pSDG1 holds after the step to the pressure-CG tolerance: the
    discrete divergence of U^{n+1} equals theta A' P^{n+1} - b."""
    o = _oracle(2, (6, 5), 3, nu=0.05, theta=0.51, dt=0.01)
    Us, P = _tg_state(o)
    rng = np.random.default_rng(5)
    Us = [U + 0.01 * rng.standard_normal(o.shape) for U in Us]
    Un, Pn, info = o.step(Us, P)
    assert info["p_converged"]
    div0 = np.linalg.norm(o.divergence(Us))
    div1 = np.linalg.norm(o.divergence(Un))
    assert div1 <= 1e-10 * div0


def test_step_theta_invariance():
    """Reading R1, derived: A' q = -div(U*) does not depend on theta, so
    U^{n+1} is the same for theta = 0.51 and theta = 1 (up to CG tolerance)."""
    outs = []
    for th in (0.51, 1.0):
        o = _oracle(2, (5, 4), 2, nu=0.02, theta=th, dt=0.02)
        o.rtol_p = 1e-14
        Us, P = _tg_state(o)
        Un, _, _ = o.step(Us, P)
        outs.append(Un)
    for a, b in zip(*outs):
        assert np.abs(a - b).max() <= 1e-11


def test_step_3d_divergence_free():
    o = _oracle(3, (3, 3, 4), 2, nu=0.01, theta=0.55, dt=0.01)
    X, Y, Z = o.coords(None)
    Us = []
    for d in range(3):
        c = o.coords(d)
        Us.append(si.taylor_green_3d(*c)[d])
    P = si.taylor_green_3d(X, Y, Z)[3]
    P = P - o.physical_mean(P)
    Un, Pn, info = o.step(Us, P)
    assert info["p_converged"]
    assert np.linalg.norm(o.divergence(Un)) <= 1e-10 * np.linalg.norm(o.divergence(Us)) + 1e-13
    assert abs(o.physical_mean(Pn)) < 1e-13


def _golden_tg():
    rows = []
    with open(os.path.join(GOLDEN, "taylor_green_2d.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(float(v) for v in line.split()))
    return rows


def test_tg_kinetic_energy_decay():
    """2D Taylor-Green (Sec. 3.4.2), 8x8 cells, N = 3, nu = 0.1, theta = 0.51,
    dt = 0.01, 10 steps: K(t = 0.1) matches the exact K0 e^{-4 nu t} to 1e-3
    (the fractional step splits viscosity and pressure, first order in dt)."""
    o = _oracle(2, (8, 8), 3, nu=0.1, theta=0.51, dt=0.01)
    Us, P = _tg_state(o)
    rows = _golden_tg()
    K0 = o.kinetic_energy(Us)
    assert abs(K0 - rows[0][2]) < 1e-10
    for _ in range(10):
        Us, P, info = o.step(Us, P)
        assert info["p_converged"]
    K = o.kinetic_energy(Us)
    assert abs(K - rows[1][2]) / rows[1][2] < 1e-3


def _l2_velocity_error(o, U, Ue):
    """sqrt(int |u_h - u|^2) over the domain, GL quadrature on each dual grid."""
    cv = float(np.prod(o.g.dx))
    return math.sqrt(sum(cv * float(np.sum(o.mass_all((U[d] - Ue[d]) ** 2))) for d in range(o.dim)))


@pytest.mark.parametrize("N,cells,min_order", [(2, (8, 16, 32), 2.5), (3, (4, 8, 16), 2.75),
                                               (4, (8, 16, 32), 4.5), (5, (4, 8), 5.5)])
def test_step_convergence_order(N, cells, min_order):
    """Spatial convergence of the whole step on the viscous 2D Taylor-Green
    vortex (exact solution of Sec. 3.4.2): nu = 0.05, theta = 0.5, L2 velocity
    error at T = 0.02 on refined grids.  The fractional step is first order in
    dt (Sec. 2.3); Richardson extrapolation 2 U(dt/2) - U(dt) with dt = 1e-3
    removes that error, so what remains is the spatial one.

    Even N and N = 5 converge at order N + 1 (measured: N = 2: 3.2, 3.7;
    N = 4: 4.8, 5.8; N = 5: 6.0), asserted >= N + 1/2.  N = 3 converges at
    order N (measured 3.2, 3.0): already the discrete divergence-free
    projection of the interpolated initial field moves it by O(h^N) for this
    degree, while the round trip of the L2 projections of Eqs.
    l2forward / l2backward alone is O(h^{N+1}).  The paper's own Taylor-Green
    convergence table (Table TGV2D, space-time version of the same spatial
    scheme) shows the same pattern: 3.26-3.28 for N = M = 3 against 3.6-3.9
    for N = M = 2 and 5.9-6.3 for N = M = 4.  A dropped order fails every
    case."""
    errs = []
    T = 0.02
    for n in cells:
        sols = []
        for dt in (1e-3, 5e-4):
            o = _oracle(2, (n, n), N, nu=0.05, theta=0.5, dt=dt)
            Us, P = _tg_state(o)
            for _ in range(int(round(T / dt))):
                Us, P = o.step_exact(Us, P)
            sols.append(Us)
        Ue, _ = _tg_state(o, T)
        errs.append(_l2_velocity_error(o, [2.0 * sols[1][d] - sols[0][d] for d in range(2)], Ue))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) >= min_order, (errs, orders)


# ------------------------------------------------------------------ exact periodic solves
@pytest.mark.parametrize("dim,n,N", [(2, (5, 4), 3), (2, (4, 6), 2), (3, (3, 4, 2), 1), (3, (2, 3, 4), 2)])
def test_block_circulant_solve_matches_dense(dim, n, N):
    """The exact Fourier solve of the periodic system equals the dense
    pseudo-inverse solution plus the kernel part of x0 (pressure, Eq. pSyst)
    and the dense solve of the SPD viscous system (Eq. implicitviscosity)."""
    o = _oracle(dim, n, N, L=(1.0, 1.4, 0.8)[:dim])
    A = o.dense(o.pressure_apply)
    ev, V = np.linalg.eigh(A)
    ker = np.abs(ev) < 1e-11 * ev.max()
    K = V[:, ker]
    rng = np.random.default_rng(1)
    b = o.pressure_apply(rng.standard_normal(o.shape)).ravel()
    x0 = rng.standard_normal(o.ndof)
    inv = np.where(ker, 0.0, 1.0 / np.where(ker, 1.0, ev))
    ref = K @ (K.T @ x0) + V @ (inv * (V.T @ b))
    x = o.pressure_solve_exact(b.reshape(o.shape), x0.reshape(o.shape)).ravel()
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)
    # kernel patterns of the oracle span exactly the numerical kernel
    Kp = o.kernel_patterns()
    assert Kp.shape[0] == ker.sum()
    Av = o.dense(o.viscous_apply)
    bv = rng.standard_normal(o.ndof)
    xv = o.viscous_solve_exact(bv.reshape(o.shape)).ravel()
    assert np.linalg.norm(xv - np.linalg.solve(Av, bv)) <= 1e-12 * np.linalg.norm(xv)


def test_exact_solve_reaches_fp64_floor():
    """Eq. pSyst on 32x32 cells at N = 7 (the benchmark degree): for a range
    right-hand side b = theta A' z the exact solve returns the range part of z
    to 3e-13 (the rounding of b itself costs about 1e-13 here), and its
    residual equals, within 1.5x, the residual that rounding the exact
    solution to FP64 leaves by itself: theta A' applied to a random
    perturbation of +-ulp(x)/(2 sqrt 3) per entry (the root mean square of a
    rounding error).  Without its residual corrections the Fourier solve
    leaves more than 4x that residual (and the gap grows with the grid)."""
    o = _oracle(2, (32, 32), 7, nu=1e-3, theta=0.51, dt=2e-3, L=(2 * math.pi, 2 * math.pi))
    X, Y = o.coords(None)
    z = np.cos(X) * np.cos(2 * Y) + 0.3 * np.sin(3 * X + 1.0) * np.cos(5 * Y)
    z = z - o.kernel_part(z)
    b = o.pressure_apply(z)
    b = b - o.kernel_part(b)
    nb = np.linalg.norm(b)
    s = np.random.default_rng(5).choice([-1.0, 1.0], size=b.shape)
    for refine, ok in ((2, True), (0, False)):
        x = o.block_circulant_solve(b, np.zeros_like(b), 0.0, o.theta, refine=refine)
        fwd = np.linalg.norm(x - z) / np.linalg.norm(z)
        r = b - o.pressure_apply(x)
        res = np.linalg.norm(r - o.kernel_part(r)) / nb
        floor = np.linalg.norm(o.pressure_apply(0.5 * np.spacing(np.abs(x)) * s / math.sqrt(3.0))) / nb
        if ok:
            assert fwd <= 3e-13, fwd
            assert res <= 1.5 * floor, (res, floor)
        else:
            assert res > 4 * floor, (fwd, res, floor)


@pytest.mark.parametrize("N,odd", [(5, True), (4, False)])
def test_pressure_sensitivity_to_operator_rounding(N, odd):
    """How precisely FP64 fixes the pressure of a step: perturb the 1D blocks
    H^R, H^L = (H^R)^T and H^C (after Eq. pSyst) by a random symmetric amount
    of 1e-15 of their size (a few units in the last place, the size of the
    rounding any FP64 evaluation of them carries) and step a perturbed
    Taylor-Green field on 32x32 cells with both systems solved exactly.  The
    velocity moves by < 1e-13.  For odd N the pressure moves by > 3e-12
    (measured 1.1e-11 here, 2.2e-10 on 64x64 cells at N = 7): its
    near-kernel modes, per-cell sawtooth patterns modulated by smooth
    envelopes (the kernel of Sec. 2.1 is larger than the constants for odd
    N), have small eigenvalues that such rounding shifts noticeably, and
    they hardly enter the gradient that updates the velocity.  For even N
    (kernel: the constants) it moves by < 1e-12 (measured 3.8e-13).  Two
    independent FP64 implementations of the step therefore agree in velocity
    to round-off but, for odd N on large grids, in pressure only to this
    sensitivity."""
    o = _oracle(2, (32, 32), N, nu=1e-3, theta=0.51, dt=2e-3, L=(2 * math.pi, 2 * math.pi))
    modes = si.stream_modes(0, 32, 8, 1e-2)
    Xu, Yu = o.coords(0)
    Xv, Yv = o.coords(1)
    X, Y = o.coords(None)
    U = [si.taylor_green_2d(Xu, Yu)[0] + si.perturbation_velocity(modes, Xu, Yu)[0],
         si.taylor_green_2d(Xv, Yv)[1] + si.perturbation_velocity(modes, Xv, Yv)[1]]
    P = si.taylor_green_2d(X, Y)[2]
    U1, P1 = o.step_exact([u.copy() for u in U], P.copy())
    rng = np.random.default_rng(3)
    E = rng.standard_normal(o.B.HR.shape) * 1e-15 * np.abs(o.B.HR).max()
    C = rng.standard_normal(o.B.HC.shape) * 1e-15 * np.abs(o.B.HC).max()
    o.B.HR = o.B.HR + E
    o.B.HL = o.B.HL + E.T
    o.B.HC = o.B.HC + 0.5 * (C + C.T)
    U2, P2 = o.step_exact([u.copy() for u in U], P.copy())
    du = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(U1, U2)))
    du /= math.sqrt(sum(float(np.sum(a * a)) for a in U1))
    dp = np.linalg.norm(P1 - P2) / np.linalg.norm(P1)
    assert du < 1e-13, du
    if odd:
        assert dp > 3e-12, dp
    else:
        assert dp < 1e-12, dp


def test_exact_step_matches_cg_step():
    """step_exact (both systems solved exactly) equals step with CG run to
    1e-14 on a small grid."""
    o = _oracle(2, (6, 5), 3, nu=0.05, theta=0.55, dt=0.01)
    o.rtol_p = o.rtol_v = 1e-14
    Us, P = _tg_state(o)
    U1, P1, _ = o.step(Us, P)
    U2, P2 = o.step_exact(Us, P)
    for a, c in zip(U1, U2):
        assert np.linalg.norm(a - c) <= 1e-11 * np.linalg.norm(c)
    assert np.linalg.norm(P1 - P2) <= 1e-10 * np.linalg.norm(P2)
