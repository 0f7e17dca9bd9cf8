"""Plain FP64 CPU oracle of the spectral semi-implicit staggered DG scheme
(Fambri & Dumbser, "Spectral semi-implicit and space-time discontinuous
Galerkin methods for the incompressible Navier-Stokes equations on staggered
Cartesian grids", Sec. 2).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  It shares no code with
the CUDA library: every matrix is recomputed here from its defining integral
and every operator is applied with whole-array numpy steps that follow the
equations term by term (no blocking, no fusion).

Layout of a field on an Nx x Ny (x Nz) periodic grid with degree N
(n1 = N + 1 nodes per direction): numpy array of shape
    2D: (Ny, Nx, n1[l2], n1[l1])          3D: (Nz, Ny, Nx, n1[l3], n1[l2], n1[l1])
in C order, i.e. element-major with the x node index fastest.  A velocity
component u_d lives on the dual grid shifted by +1/2 in direction d: the block
stored at element index i (along d) is the dual cell i+1/2.

Readings of points the paper leaves open (each is exercised by a test):
  R1  pressure unknown: theta * A' P^{n+1} = b_U - (1 - theta) A' P^n
      (Eq. pSyst), q = theta P^{n+1} + (1 - theta) P^n used in Eq. LOvelocityU.
  R2  periodic wrap for every cell (the 1D periodic derivation, Eq. pSyst1d).
  R3  singular periodic system: b is projected to zero Euclidean mean; after
      each solve P^{n+1} is shifted to zero physical mean.
  R4  H is the SUM over directions of (theta dt / dx_d^2) M^{perp d} H_d.
  R5  Eq. Uy/Uz index typo read as U_{i,j+1,k}, U_{i,j,k+1}.
  R6  viscous operator: M^{xyz} + nu dt sum_d (1/dx_d^2) M^{perp d} H_d,
      right-hand side M^{xyz} Fu (Eqs. uSDG12, Ux-Uz, implicitviscosity).
  R7  Rusanov speed on a face normal to d: s = 2 max(|v_d^+|, |v_d^-|),
      pointwise at face nodes; the viscous part of s is dropped because
      viscosity is implicit.
  R8  nonlinear terms by collocation at the n1 Gauss-Legendre nodes.
  R9  SSP-RK3 (Shu-Osher form) on the convective operator only.
  R10 initial data: point values at the element's own GL nodes.
  R11 CG: Hestenes-Stiefel, Euclidean norm, stop on the recursive residual
      ||r_k|| <= rtol ||b||, x0 = P^n (pressure) / Fu (viscous).
  R12 a time step above the explicit limit of Eq. CFL1 (CFL >= 1) keeps its
      dt for the implicit solves and advances the explicit convection in
      nsub equal SSP-RK3 sub-steps of dt / nsub (nsub = 1: the scheme as
      stated; otherwise nsub >= CFL / 0.5).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "gauss_legendre_01", "lagrange", "lagrange_deriv", "Basis", "Grid",
    "Oracle", "cg", "CGResult",
]


# =====================================================================  Sec. 2.1
def gauss_legendre_01(n1: int):
    """Gauss-Legendre nodes and weights mapped to [0, 1] (Sec. 2.1: the basis
    is the Lagrange interpolant through these points).  Weights sum to 1."""
    x, w = np.polynomial.legendre.leggauss(n1)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(nodes: np.ndarray, p: int, x):
    """phi_p(x) = prod_{q != p} (x - xi_q) / (xi_p - xi_q)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for q in range(len(nodes)):
        if q != p:
            out = out * (x - nodes[q]) / (nodes[p] - nodes[q])
    return out


def lagrange_deriv(nodes: np.ndarray, p: int, x):
    """phi_p'(x) by the product rule applied to `lagrange`."""
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    out = np.zeros_like(x)
    for m in range(n):
        if m == p:
            continue
        term = np.ones_like(x) / (nodes[p] - nodes[m])
        for q in range(n):
            if q != p and q != m:
                term = term * (x - nodes[q]) / (nodes[p] - nodes[q])
        out = out + term
    return out


def _integrate01(f, nq: int):
    """Integral of f over [0, 1] by an nq-point Gauss-Legendre rule."""
    s, w = gauss_legendre_01(nq)
    return float(np.sum(w * f(s)))


class Basis:
    """1D reference-element matrices of degree N (Sec. 2.1, Eq. matrices;
    Sec. 2.2, the L2 projections M^L, M^R), each computed from its integral.

    Attributes (n1 x n1 unless noted):
      xi, w         GL nodes / weights on [0, 1]                   (n1,)
      M             mass matrix int phi_p phi_q
      Rt, Lt        R~, L~ of Eq. matrices (weak gradient, dual cell)
      Rb, Lb        R-bar, L-bar of Eq. matrices (weak divergence, main cell)
      ML, MR        M^L, M^R of the L2 projections (Sec. 2.2)
      HR, HL, HC    H^R = -Rb M^-1 Rt, H^L = -Lb M^-1 Lt,
                    H^C = Rb M^-1 Lt + Lb M^-1 Rt            (after Eq. pSyst)
      Dn            nodal derivative Dn[k, m] = phi_m'(xi_k)
      phi0, phi1    phi_m(0), phi_m(1)                               (n1,)
    """

    def __init__(self, N: int):
        if N < 0:
            raise ValueError("N must be >= 0")
        self.N = N
        n1 = N + 1
        self.n1 = n1
        xi, w = gauss_legendre_01(n1)
        self.xi, self.w = xi, w
        nq = n1 + 3  # exact for the degree <= 2N integrands below

        def phi(p, x):
            return lagrange(xi, p, x)

        def dphi(p, x):
            return lagrange_deriv(xi, p, x)

        Z = lambda: np.zeros((n1, n1))
        M, Rt, Lt, Rb, Lb, ML, MR = Z(), Z(), Z(), Z(), Z(), Z(), Z()
        for p in range(n1):
            for q in range(n1):
                M[p, q] = _integrate01(lambda s: phi(p, s) * phi(q, s), nq)
                Rt[p, q] = (phi(p, 0.5) * phi(q, 0.0)
                            + 0.5 * _integrate01(
                                lambda s: phi(p, 0.5 + 0.5 * s) * dphi(q, 0.5 * s), nq))
                Lt[p, q] = (phi(p, 0.5) * phi(q, 1.0)
                            - 0.5 * _integrate01(
                                lambda s: phi(p, 0.5 * s) * dphi(q, 0.5 + 0.5 * s), nq))
                Rb[p, q] = (phi(p, 1.0) * phi(q, 0.5)
                            - 0.5 * _integrate01(
                                lambda s: dphi(p, 0.5 + 0.5 * s) * phi(q, 0.5 * s), nq))
                Lb[p, q] = (phi(p, 0.0) * phi(q, 0.5)
                            + 0.5 * _integrate01(
                                lambda s: dphi(p, 0.5 * s) * phi(q, 0.5 + 0.5 * s), nq))
                ML[p, q] = 0.5 * _integrate01(
                    lambda s: phi(p, 0.5 * s) * phi(q, 0.5 + 0.5 * s), nq)
                MR[p, q] = 0.5 * _integrate01(
                    lambda s: phi(p, 0.5 + 0.5 * s) * phi(q, 0.5 * s), nq)
        self.M, self.Rt, self.Lt, self.Rb, self.Lb = M, Rt, Lt, Rb, Lb
        self.ML, self.MR = ML, MR
        Minv = np.linalg.inv(M)
        self.Minv = Minv
        self.HR = -(Rb @ Minv @ Rt)
        self.HL = -(Lb @ Minv @ Lt)
        self.HC = Rb @ Minv @ Lt + Lb @ Minv @ Rt
        self.Dn = np.array([[dphi(m, xi[k]) for m in range(n1)] for k in range(n1)])
        self.phi0 = np.array([float(phi(m, 0.0)) for m in range(n1)])
        self.phi1 = np.array([float(phi(m, 1.0)) for m in range(n1)])


# =====================================================================  grids
@dataclasses.dataclass
class Grid:
    """Periodic box [0, L_x] x [0, L_y] (x [0, L_z]) split into n cells per
    direction (Sec. 2.1: main cells T_{i,j,k} and dual cells T_{i+1/2,j,k}...)."""
    dim: int
    n: tuple
    L: tuple

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)[: self.dim]
        self.L = tuple(float(v) for v in self.L)[: self.dim]
        if len(self.n) != self.dim or len(self.L) != self.dim:
            raise ValueError("n and L need one entry per dimension")

    @property
    def dx(self):
        return tuple(self.L[d] / self.n[d] for d in range(self.dim))

    @property
    def ncell(self):
        return int(np.prod(self.n))


# =====================================================================  CG
@dataclasses.dataclass
class CGResult:
    x: np.ndarray
    iters: int
    rel_res: float
    converged: bool


def cg(apply, b: np.ndarray, x0: np.ndarray, rtol: float, maxit: int = 20000) -> CGResult:
    """Unpreconditioned conjugate gradients (Hestenes-Stiefel), the solver the
    paper uses for the pressure and viscous systems (Sec. 2.1, after
    Eq. weakgradient).  Stops when ||r_k||_2 <= rtol ||b||_2 on the recursive
    residual; returns x0 unchanged if ||b|| = 0."""
    x = x0.astype(np.float64).copy()
    bnorm = float(np.sqrt(np.dot(b.ravel(), b.ravel())))
    if bnorm == 0.0:
        return CGResult(x, 0, 0.0, True)
    r = b - apply(x)
    p = r.copy()
    rr = float(np.dot(r.ravel(), r.ravel()))
    it = 0
    while it < maxit and math.sqrt(rr) > rtol * bnorm:
        Ap = apply(p)
        pAp = float(np.dot(p.ravel(), Ap.ravel()))
        if not pAp > 0.0:
            break
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.dot(r.ravel(), r.ravel()))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
    rel = math.sqrt(rr) / bnorm
    return CGResult(x, it, rel, rel <= rtol)


# =====================================================================  scheme
class Oracle:
    """The semi-implicit staggered DG scheme of Sec. 2 on a periodic grid.

    Parameters follow the problem statement: grid, degree N, viscosity nu,
    implicitness theta (Sec. 2.1, P^{n+theta}), time step dt.
    """

    def __init__(self, grid: Grid, N: int, nu: float, theta: float, dt: float,
                 rtol_p: float = 1e-12, rtol_v: float = 1e-12, maxit: int = 20000,
                 nsub: int = 1):
        if grid.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.g = grid
        self.dim = grid.dim
        self.N = N
        self.n1 = N + 1
        self.nu, self.theta, self.dt = float(nu), float(theta), float(dt)
        self.rtol_p, self.rtol_v, self.maxit = rtol_p, rtol_v, maxit
        if int(nsub) < 1:
            raise ValueError("nsub must be >= 1")
        self.nsub = int(nsub)
        self.B = Basis(N)

    # ------------------------------------------------------------- layout
    @property
    def shape(self):
        n = self.g.n
        lead = tuple(reversed(n))  # (Nz,) Ny, Nx
        return lead + (self.n1,) * self.dim

    @property
    def ndof(self):
        return int(np.prod(self.shape))

    def _eax(self, d):
        """Array axis of the element index along direction d."""
        return self.dim - 1 - d

    def _lax(self, d):
        """Array axis of the local node index along direction d."""
        return 2 * self.dim - 1 - d

    def nodes(self, d, dual: bool):
        """Physical coordinate along direction d of every DOF, broadcastable to
        the field shape.  Main cell i spans [i dx, (i+1) dx]; the dual cell
        i+1/2 spans [(i+1/2) dx, (i+3/2) dx] (Sec. 2.1: x_{i+1/2} are the main
        cell faces, x_i the centres)."""
        dx = self.g.dx[d]
        i = np.arange(self.g.n[d], dtype=np.float64)
        off = 0.5 if dual else 0.0
        c = (i[:, None] + off + self.B.xi[None, :]) * dx  # c[i, l]
        shp = [1] * (2 * self.dim)
        shp[self._eax(d)] = self.g.n[d]
        shp[self._lax(d)] = self.n1
        return c.reshape(shp)  # element axis precedes local axis

    def coords(self, dual_dir=None):
        """Tuple of coordinate arrays (x, y[, z]) broadcast to the field shape,
        for the main grid (dual_dir None) or the dual grid of direction d."""
        out = []
        for d in range(self.dim):
            out.append(np.broadcast_to(self.nodes(d, dual_dir == d), self.shape))
        return tuple(out)

    # ------------------------------------------------------------- 1D tools (Eq. tensorP1)
    def along(self, Z, X, d):
        """Z^d . X: apply the n1 x n1 matrix Z along the local index of
        direction d (Eq. tensorP1)."""
        ax = self._lax(d)
        Xm = np.moveaxis(X, ax, -1)
        Y = Xm @ Z.T
        return np.moveaxis(Y, -1, ax)

    def shift(self, X, d, s):
        """Periodic element shift: returns Y with Y[i] = X[i - s] along d."""
        return np.roll(X, s, axis=self._eax(d))

    def mass_perp(self, X, d):
        """M^{perp d} . X: diagonal mass along every direction except d."""
        Y = X
        for e in range(self.dim):
            if e != d:
                Y = self.along(self.B.M, Y, e)
        return Y

    def mass_all(self, X):
        """M^{xyz} . X: diagonal reference mass along every direction."""
        Y = X
        for e in range(self.dim):
            Y = self.along(self.B.M, Y, e)
        return Y

    # ------------------------------------------------------------- Eq. pSyst
    def H_dir(self, X, d):
        """(H^L X_{i-1} + H^C X_i + H^R X_{i+1}) along direction d."""
        B = self.B
        return (self.along(B.HL, self.shift(X, d, +1), d)
                + self.along(B.HC, X, d)
                + self.along(B.HR, self.shift(X, d, -1), d))

    def Aprime(self, X):
        """A' X = dt sum_d (1/dx_d^2) M^{perp d} H_d X (Eq. pSyst without theta)."""
        Y = np.zeros_like(X)
        for d in range(self.dim):
            Y = Y + (self.dt / self.g.dx[d] ** 2) * self.mass_perp(self.H_dir(X, d), d)
        return Y

    def pressure_apply(self, X):
        """Left-hand side of Eq. pSyst: theta A' X."""
        return self.theta * self.Aprime(X)

    def viscous_apply(self, X):
        """(M + nu H) X of Eq. implicitviscosity with the scales of Eqs.
        uSDG12 and Ux-Uz: M^{xyz} X + nu dt sum_d (1/dx_d^2) M^{perp d} H_d X."""
        return self.mass_all(X) + self.nu * self.Aprime(X)

    # ------------------------------------------------------------- Eq. weakgradient, pSDG1
    def weak_gradient(self, P, d):
        """(D_d P)_{i+1/2} = R~ P_{i+1} - L~ P_i (Eq. weakgradient), stored at
        dual index i."""
        return self.along(self.B.Rt, self.shift(P, d, -1), d) - self.along(self.B.Lt, P, d)

    def weak_divergence(self, U, d):
        """R-bar U_{i+1/2} - L-bar U_{i-1/2} along d (the bracket of Eq. pSDG1)."""
        return self.along(self.B.Rb, U, d) - self.along(self.B.Lb, self.shift(U, d, +1), d)

    def divergence(self, Us):
        """Left-hand side of Eq. pSDG1: sum_d (1/dx_d) M^{perp d} (Rb U - Lb U)_d."""
        out = np.zeros(self.shape)
        for d in range(self.dim):
            out = out + self.mass_perp(self.weak_divergence(Us[d], d), d) / self.g.dx[d]
        return out

    def pressure_rhs(self, Us, P_old):
        """b of Eq. pSyst (reading R1): substituting U = U* - (dt/dx) M^-1 D P^{n+theta}
        into Eq. pSDG1 gives theta A' P^{n+1} = -div(U*) - (1-theta) A' P^n."""
        return -self.divergence(Us) - (1.0 - self.theta) * self.Aprime(P_old)

    def velocity_update(self, Us, q):
        """Eq. LOvelocityU-W: U_d = U*_d - (dt/dx_d) M^-1 (R~ q_{i+1} - L~ q_i)."""
        return [Us[d] - (self.dt / self.g.dx[d]) * self.along(self.B.Minv, self.weak_gradient(q, d), d)
                for d in range(self.dim)]

    # ------------------------------------------------------------- Sec. 2.2 projections
    def dual_to_main(self, U, d):
        """Eq. l2forward: U_i = M^-1 (M^L U_{i-1/2} + M^R U_{i+1/2}) along d."""
        B = self.B
        return self.along(B.Minv, self.along(B.ML, self.shift(U, d, +1), d) + self.along(B.MR, U, d), d)

    def main_to_dual(self, F, d):
        """Eq. l2backward: F_{i+1/2} = M^-1 (M^L F_i + M^R F_{i+1}) along d."""
        B = self.B
        return self.along(B.Minv, self.along(B.ML, F, d) + self.along(B.MR, self.shift(F, d, -1), d), d)

    # ------------------------------------------------------------- Sec. 2.2 convection
    def _face(self, X, d, side):
        """Trace of X on the face at xi = side (0 or 1) along d: sum_l phi_l(side) X_l."""
        vec = self.B.phi1 if side == 1 else self.B.phi0
        return np.tensordot(X, vec, axes=([self._lax(d)], [0]))

    def _lift(self, f, d, side):
        """Outer product of a face array with phi_m(side) along direction d."""
        vec = self.B.phi1 if side == 1 else self.B.phi0
        return np.moveaxis(f[..., None] * vec, -1, self._lax(d))

    def convection(self, V):
        """Explicit DG convective operator L(V) on the main grid (Eqs. Fu-Fw with
        the Rusanov flux; readings R7, R8):
            L(q) = - sum_d (1/dx_d) M_d^-1 [phi(1) F^_{i+1/2} - phi(0) F^_{i-1/2}
                                           - Dn^T W (q v_d)]
        for every component q of V = (u, v[, w])."""
        B = self.B
        out = [np.zeros(self.shape) for _ in range(self.dim)]
        DW = B.Dn.T @ np.diag(B.w)  # (DW)[m, k] = phi_m'(xi_k) w_k
        for d in range(self.dim):
            vd = V[d]
            # face i+1/2: "-" trace from cell i (xi = 1), "+" trace from cell i+1 (xi = 0)
            vd_R = self._face(vd, d, 1)
            vd_Lp = np.roll(self._face(vd, d, 0), -1, axis=self._eax(d))
            s = 2.0 * np.maximum(np.abs(vd_R), np.abs(vd_Lp))
            for c in range(self.dim):
                q = V[c]
                flux_vol = q * vd
                qm = self._face(q, d, 1)
                qp = np.roll(self._face(q, d, 0), -1, axis=self._eax(d))
                fhat = 0.5 * (qm * vd_R + qp * vd_Lp) - 0.5 * s * (qp - qm)  # at face i+1/2
                fhat_left = np.roll(fhat, 1, axis=self._eax(d))             # face i-1/2
                surf = self._lift(fhat, d, 1) - self._lift(fhat_left, d, 0)
                vol = self.along(DW, flux_vol, d)
                out[c] = out[c] - self.along(B.Minv, surf - vol, d) / self.g.dx[d]
        return out

    def rk3(self, V):
        """Third-order SSP Runge-Kutta (Shu-Osher form) on dV/dt = L(V) over one
        dt (reading R9), taken in nsub equal sub-steps (reading R12)."""
        k = self.dt / self.nsub
        for _ in range(self.nsub):
            L0 = self.convection(V)
            V1 = [V[c] + k * L0[c] for c in range(self.dim)]
            L1 = self.convection(V1)
            V2 = [0.75 * V[c] + 0.25 * (V1[c] + k * L1[c]) for c in range(self.dim)]
            L2 = self.convection(V2)
            V = [V[c] / 3.0 + (2.0 / 3.0) * (V2[c] + k * L2[c]) for c in range(self.dim)]
        return V

    # ------------------------------------------------------------- gauge (reading R3)
    def physical_mean(self, P):
        """(1/|Omega|) int p dx = (1/ncell) sum_cells sum_l W_l p_l."""
        return float(np.sum(self.mass_all(P))) / self.g.ncell

    # ------------------------------------------------------------- Sec. 2.3, compact scheme
    def step(self, Us, P):
        """One time step of the compact fractional-step scheme
        (Eqs. LOdiffusionU-W, LOpressure, LOvelocityU-W):
          1. project each u_d from its dual grid to the main grid (Eq. l2forward)
          2. SSP-RK3 of the explicit convection on the main grid   (Eq. Fu-Fw)
          3. implicit viscosity (M + nu H) U = M Fu per component   (CG)
          4. project back to the dual grids                         (Eq. l2backward)
          5. pressure system theta A' P^{n+1} = b                   (CG, R1, R3)
          6. velocity update with q = theta P^{n+1} + (1-theta) P^n
        Returns (U_new list, P_new, info dict)."""
        V = [self.dual_to_main(Us[d], d) for d in range(self.dim)]
        F = self.rk3(V)
        Vh, vit = [], []
        for c in range(self.dim):
            res = cg(self.viscous_apply, self.mass_all(F[c]), F[c], self.rtol_v, self.maxit)
            Vh.append(res.x)
            vit.append(res.iters)
        Ustar = [self.main_to_dual(Vh[d], d) for d in range(self.dim)]
        b = self.pressure_rhs(Ustar, P)
        b = b - np.mean(b)
        res = cg(self.pressure_apply, b, P, self.rtol_p, self.maxit)
        Pn = res.x - self.physical_mean(res.x)
        q = self.theta * Pn + (1.0 - self.theta) * P
        Un = self.velocity_update(Ustar, q)
        info = dict(p_iters=res.iters, p_rel_res=res.rel_res, p_converged=res.converged,
                    v_iters=vit, bnorm=float(np.linalg.norm(b)))
        return Un, Pn, info

    # ------------------------------------------------------------- Sec. 2.5 diagnostics
    def kinetic_energy(self, Us):
        """K = (1/|Omega|) int |v|^2 / 2 dx, each component integrated with GL
        quadrature on its own dual grid."""
        vol = float(np.prod(self.g.L))
        cellvol = float(np.prod(self.g.dx))
        tot = 0.0
        for d in range(self.dim):
            tot += 0.5 * cellvol * float(np.sum(self.mass_all(Us[d] * Us[d])))
        return tot / vol

    # ------------------------------------------------------------- exact periodic solves
    def kernel_patterns(self):
        """Orthonormal local patterns (rows) whose repetition in every element
        spans the kernel of the periodic pressure operator: tensor products of
        a basis of null(R~ - L~) (Sec. 2.1: weak solutions of grad p = 0)."""
        G = self.B.Rt - self.B.Lt
        _, sv, vt = np.linalg.svd(G)
        tol = 1e-10 * max(1.0, np.abs(self.B.Rt).max())
        null1 = vt[sv <= tol]  # rows: orthonormal basis of null(G)
        pats = []
        for idx in itertools.product(range(null1.shape[0]), repeat=self.dim):
            p = np.ones(())
            for d in reversed(range(self.dim)):  # local axes ordered (l_{dim-1}, ..., l_0)
                p = np.multiply.outer(p, null1[idx[d]])
            pats.append(p.reshape(-1))
        return np.array(pats)

    def kernel_part(self, X):
        """Euclidean projection of X onto the kernel (element-repeated
        patterns of kernel_patterns)."""
        K = self.kernel_patterns()
        npe = self.n1 ** self.dim
        Xe = X.reshape(-1, npe)
        coef = K @ Xe.sum(axis=0) / Xe.shape[0]
        return np.broadcast_to(K.T @ coef, Xe.shape).reshape(X.shape)

    def _symbols(self, d):
        """W^{-1/2} (H^L e^{-ik} + H^C + H^R e^{ik}) W^{-1/2} eigen-decomposed
        for every wavenumber k = 2 pi m / n_d (numpy FFT ordering)."""
        B = self.B
        n = self.g.n[d]
        ws = 1.0 / np.sqrt(B.w)
        lam, vec = [], []
        for m in range(n):
            k = 2.0 * math.pi * m / n
            S = B.HL * np.exp(-1j * k) + B.HC + B.HR * np.exp(1j * k)
            S = 0.5 * (S + S.conj().T)
            e, V = np.linalg.eigh(ws[:, None] * S * ws[None, :])
            lam.append(e)
            vec.append(V)
        return np.array(lam), np.array(vec)  # (n, n1), (n, n1, n1)

    def block_circulant_solve(self, b, x0, cmass, scale, raw=False, refine=2):
        """Exact solution of (cmass M^{xyz} + scale * A') x = b on the periodic
        grid, A' = dt sum_d (1/dx_d^2) M^{perp d} H_d (Eq. pSyst).  The operator
        is block-circulant: a discrete Fourier transform over the elements of
        each direction turns it into one n1^dim x n1^dim Hermitian block per
        wave vector, W^{1/2} [cmass I + sum_d scale dt/dx_d^2 (S_d(k_d) in
        direction d)] W^{1/2} with S_d = W^{-1/2} (H^L e^{-ik} + H^C +
        H^R e^{ik}) W^{-1/2}, which the 1D eigenvectors of the S_d
        diagonalise.  Zero eigenvalues (the kernel, cmass = 0) are dropped and
        the kernel part of x0 is kept, as CG from x0 does (raw: the spectral
        solution itself, W-orthogonal to the kernel, is returned; this map is
        symmetric, the projected one is not).

        The Fourier solve alone carries the rounding of its transforms into
        every mode, which the ill-conditioned pressure system turns into a
        relative solution error of about 4e-11 on 128^2 cells at N = 7; each
        of the `refine` residual corrections x += S (b - A x), with S the
        spectral inverse and A the operator applied term by term, brings the
        solution to the accuracy FP64 can represent (its residual then equals
        the residual that rounding the exact solution to FP64 leaves)."""
        def op(X):
            Y = scale * self.Aprime(X)
            return Y + cmass * self.mass_all(X) if cmass != 0.0 else Y
        x = self._spectral_inverse(b, cmass, scale)
        for _ in range(refine):
            x = x + self._spectral_inverse(b - op(x), cmass, scale)
        if cmass == 0.0 and not raw:
            x = x - self.kernel_part(x) + self.kernel_part(x0)
        return x

    def _spectral_inverse(self, b, cmass, scale):
        """One Fourier-space solve of block_circulant_solve (kernel dropped)."""
        dim = self.dim
        eax = [self._eax(d) for d in range(dim)]
        lax = [self._lax(d) for d in range(dim)]
        w = self.B.w
        sq = np.sqrt(w)
        # D^{-1} = W^{-1/2} in every direction
        Bh = np.fft.fftn(b, axes=eax)
        for d in range(dim):
            shp = [1] * (2 * dim)
            shp[lax[d]] = self.n1
            Bh = Bh / sq.reshape(shp)
        syms = [self._symbols(d) for d in range(dim)]
        # transform to the eigenbasis of each direction (per wavenumber)
        def along_batched(X, V, d, conj):
            # X[..., e_d, ..., l_d, ...]; V[e_d] is (n1 x n1): X_l <- sum_k M[e][l][k] X_k
            Xm = np.moveaxis(np.moveaxis(X, eax[d], 0), lax[d] if lax[d] > eax[d] else lax[d] + 1, -1)
            M = V.conj().transpose(0, 2, 1) if conj else V  # (n, n1, n1)
            shp = (M.shape[0],) + (1,) * (Xm.ndim - 2) + M.shape[1:]
            Y = np.einsum('e...k,e...lk->e...l', Xm, M.reshape(shp))
            Y = np.moveaxis(Y, -1, lax[d] if lax[d] > eax[d] else lax[d] + 1)
            return np.moveaxis(Y, 0, eax[d])
        Y = Bh
        for d in range(dim):
            Y = along_batched(Y, syms[d][1], d, conj=True)
        den = np.full(Y.shape, cmass, dtype=np.float64)
        for d in range(dim):
            lam = syms[d][0]  # (n_d, n1)
            shp = [1] * (2 * dim)
            shp[eax[d]] = lam.shape[0]
            shp[lax[d]] = self.n1
            den = den + scale * self.dt / self.g.dx[d] ** 2 * lam.reshape(shp)
        tol = 1e-11 * np.abs(den).max()
        Y = np.where(np.abs(den) > tol, Y / np.where(np.abs(den) > tol, den, 1.0), 0.0)
        for d in range(dim):
            Y = along_batched(Y, syms[d][1], d, conj=False)
        for d in range(dim):
            shp = [1] * (2 * dim)
            shp[lax[d]] = self.n1
            Y = Y / sq.reshape(shp)
        return np.real(np.fft.ifftn(Y, axes=eax))

    def pressure_solve_exact(self, b, x0):
        """theta A' x = b solved exactly (block_circulant_solve)."""
        return self.block_circulant_solve(b, x0, 0.0, self.theta)

    def viscous_solve_exact(self, b):
        """(M + nu A') x = b solved exactly (block_circulant_solve)."""
        return self.block_circulant_solve(b, b, 1.0, self.nu)

    def step_exact(self, Us, P, intermediates=None):
        """`step` with both linear systems solved exactly instead of by CG.
        If `intermediates` is a dict, U* and b are stored in it."""
        V = [self.dual_to_main(Us[d], d) for d in range(self.dim)]
        F = self.rk3(V)
        Vh = [self.viscous_solve_exact(self.mass_all(F[c])) for c in range(self.dim)]
        Ustar = [self.main_to_dual(Vh[d], d) for d in range(self.dim)]
        b = self.pressure_rhs(Ustar, P)
        b = b - np.mean(b)
        x = self.pressure_solve_exact(b, P)
        Pn = x - self.physical_mean(x)
        q = self.theta * Pn + (1.0 - self.theta) * P
        if intermediates is not None:
            intermediates["Ustar"] = Ustar
            intermediates["b"] = b
        return self.velocity_update(Ustar, q), Pn

    # ------------------------------------------------------------- dense assembly
    def dense(self, apply):
        """Dense matrix of a linear operator on the field space, column by
        column (apply to unit vectors).  Tiny grids only."""
        n = self.ndof
        A = np.zeros((n, n))
        e = np.zeros(n)
        for k in range(n):
            e[k] = 1.0
            A[:, k] = apply(e.reshape(self.shape)).ravel()
            e[k] = 0.0
        return A
