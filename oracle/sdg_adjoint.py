"""Tangent (JVP) and adjoint (VJP) of one time step of the oracle's scheme
(Sec. 2.3, Eqs. LOdiffusionU-W, LOpressure, LOvelocityU-W), written out
stage by stage in plain numpy FP64.

TEST INFRASTRUCTURE ONLY, like `sdg_oracle`: only the test suite, the smoke
check and the benchmark's CPU legs may import it; it shares no code with the
CUDA library.

The step is the one of `Oracle.step_exact` (both linear systems solved
exactly), as a function of the dual-grid velocities U, the pressure P and the
viscosity nu:
    V_d = Pi_dm(U_d)                      (Eq. l2forward)
    F   = RK3(V)                          (Eqs. Fu-Fw, nsub sub-steps, R9, R12)
    Vh  = (M + nu A')^-1 M F              (Eq. implicitviscosity, R6)
    U*  = Pi_md(Vh)                       (Eq. l2backward)
    b   = C0 (-div U* - (1 - theta) A' P) (Eqs. pSDG1, pSyst, R1; C0 removes the mean)
    x   = (I - K) G b + K(P)              (G the spectral inverse of theta A',
                                          K the kernel part, R3)
    Pn  = x - mean_phys(x)                (gauge, R3)
    Un  = U* - (dt/dx_d) M^-1 D_d (theta Pn + (1 - theta) P)   (Eq. LOvelocityU-W)
The only non-linear stage is the Rusanov convection.  Its flux speed
s = 2 max(|v-|, |v+|) (R7) is differentiated with the sub-gradient of the
larger side (|v-| >= |v+| selects v-), sign(0) = 0.

Every transpose is the transpose with respect to the Euclidean inner product
of the DOF arrays (sum over all nodes), the one the CG solves use.
"""
from __future__ import annotations

import numpy as np

from .sdg_oracle import Oracle

__all__ = ["Adjoint"]


class Adjoint:
    def __init__(self, o: Oracle):
        self.o = o

    # ----------------------------------------------------------------- linear pieces
    def along_T(self, Z, X, d):
        return self.o.along(Z.T, X, d)

    def shift_T(self, X, d, s):
        return self.o.shift(X, d, -s)

    def dual_to_main_T(self, Y, d):
        """Transpose of Eq. l2forward: Pi_dm = Minv (ML S+ + MR)."""
        o, B = self.o, self.o.B
        Z = o.along(B.Minv, Y, d)  # Minv is diagonal
        return self.shift_T(self.along_T(B.ML, Z, d), d, +1) + self.along_T(B.MR, Z, d)

    def main_to_dual_T(self, Y, d):
        """Transpose of Eq. l2backward: Pi_md = Minv (ML + MR S-)."""
        o, B = self.o, self.o.B
        Z = o.along(B.Minv, Y, d)
        return self.along_T(B.ML, Z, d) + self.shift_T(self.along_T(B.MR, Z, d), d, -1)

    def weak_gradient_T(self, Y, d):
        """Transpose of (D_d P)_{i+1/2} = R~ P_{i+1} - L~ P_i."""
        B = self.o.B
        return self.shift_T(self.along_T(B.Rt, Y, d), d, -1) - self.along_T(B.Lt, Y, d)

    def weak_divergence_T(self, Y, d):
        """Transpose of R-bar U_{i+1/2} - L-bar U_{i-1/2}."""
        B = self.o.B
        return self.along_T(B.Rb, Y, d) - self.shift_T(self.along_T(B.Lb, Y, d), d, +1)

    def divergence_T(self, Y):
        o = self.o
        return [self.weak_divergence_T(o.mass_perp(Y, d), d) / o.g.dx[d] for d in range(o.dim)]

    def gauge_T(self, Y):
        """Transpose of x -> x - (1/ncell) sum(M^{xyz} x) 1."""
        o = self.o
        return Y - o.mass_all(np.ones(o.shape)) * (np.sum(Y) / o.g.ncell)

    # ----------------------------------------------------------------- convection
    def _faces(self, V, d, c):
        o = self.o
        qm = o._face(V[c], d, 1)
        qp = np.roll(o._face(V[c], d, 0), -1, axis=o._eax(d))
        vR = o._face(V[d], d, 1)
        vLp = np.roll(o._face(V[d], d, 0), -1, axis=o._eax(d))
        return qm, qp, vR, vLp

    @staticmethod
    def _speed_grad(vR, vLp):
        """s = 2 max(|vR|, |vLp|) and its sub-gradient (ds/dvR, ds/dvLp)."""
        left = np.abs(vR) >= np.abs(vLp)
        s = 2.0 * np.maximum(np.abs(vR), np.abs(vLp))
        return s, np.where(left, 2.0 * np.sign(vR), 0.0), np.where(left, 0.0, 2.0 * np.sign(vLp))

    def convection_jvp(self, V, dV):
        """Derivative of Oracle.convection at V in the direction dV."""
        o, B = self.o, self.o.B
        DW = B.Dn.T @ np.diag(B.w)
        out = [np.zeros(o.shape) for _ in range(o.dim)]
        for d in range(o.dim):
            for c in range(o.dim):
                qm, qp, vR, vLp = self._faces(V, d, c)
                dqm, dqp, dvR, dvLp = self._faces(dV, d, c)
                s, sR, sL = self._speed_grad(vR, vLp)
                ds = sR * dvR + sL * dvLp
                df = (0.5 * (dqm * vR + qm * dvR + dqp * vLp + qp * dvLp)
                      - 0.5 * ds * (qp - qm) - 0.5 * s * (dqp - dqm))
                df_left = np.roll(df, 1, axis=o._eax(d))
                surf = o._lift(df, d, 1) - o._lift(df_left, d, 0)
                vol = o.along(DW, dV[c] * V[d] + V[c] * dV[d], d)
                out[c] = out[c] - o.along(B.Minv, surf - vol, d) / o.g.dx[d]
        return out

    def convection_vjp(self, V, lam):
        """Transpose of convection_jvp(V, .) applied to lam."""
        o, B = self.o, self.o.B
        DW = B.Dn.T @ np.diag(B.w)
        g = [np.zeros(o.shape) for _ in range(o.dim)]
        for d in range(o.dim):
            ea = o._eax(d)
            for c in range(o.dim):
                qm, qp, vR, vLp = self._faces(V, d, c)
                s, sR, sL = self._speed_grad(vR, vLp)
                Z = -o.along(B.Minv, lam[c], d) / o.g.dx[d]
                # surf = lift(df, 1) - lift(roll(df, +1), 0)
                lf = o._face(Z, d, 1) - np.roll(o._face(Z, d, 0), -1, axis=ea)
                # vol enters with a minus sign: - along(DW, prod)
                lprod = -self.along_T(DW, Z, d)
                g[c] = g[c] + lprod * V[d]
                g[d] = g[d] + lprod * V[c]
                lqm = lf * (0.5 * vR + 0.5 * s)
                lqp = lf * (0.5 * vLp - 0.5 * s)
                jump = lf * 0.5 * (qp - qm)
                lvR = lf * 0.5 * qm - jump * sR
                lvLp = lf * 0.5 * qp - jump * sL
                g[c] = g[c] + o._lift(lqm, d, 1) + o._lift(np.roll(lqp, 1, axis=ea), d, 0)
                g[d] = g[d] + o._lift(lvR, d, 1) + o._lift(np.roll(lvLp, 1, axis=ea), d, 0)
        return g

    # ----------------------------------------------------------------- RK3
    def _rk3_states(self, V):
        """Input and stage states of every sub-step of Oracle.rk3."""
        o = self.o
        k = o.dt / o.nsub
        out = []
        W = V
        for _ in range(o.nsub):
            L0 = o.convection(W)
            S1 = [W[c] + k * L0[c] for c in range(o.dim)]
            L1 = o.convection(S1)
            S2 = [0.75 * W[c] + 0.25 * (S1[c] + k * L1[c]) for c in range(o.dim)]
            L2 = o.convection(S2)
            out.append((W, S1, S2))
            W = [W[c] / 3.0 + (2.0 / 3.0) * (S2[c] + k * L2[c]) for c in range(o.dim)]
        return out, W

    def rk3_jvp(self, V, dV):
        o = self.o
        k = o.dt / o.nsub
        W, dW = V, dV
        for _ in range(o.nsub):
            L0, dL0 = o.convection(W), self.convection_jvp(W, dW)
            S1 = [W[c] + k * L0[c] for c in range(o.dim)]
            dS1 = [dW[c] + k * dL0[c] for c in range(o.dim)]
            L1, dL1 = o.convection(S1), self.convection_jvp(S1, dS1)
            S2 = [0.75 * W[c] + 0.25 * (S1[c] + k * L1[c]) for c in range(o.dim)]
            dS2 = [0.75 * dW[c] + 0.25 * (dS1[c] + k * dL1[c]) for c in range(o.dim)]
            L2, dL2 = o.convection(S2), self.convection_jvp(S2, dS2)
            W = [W[c] / 3.0 + (2.0 / 3.0) * (S2[c] + k * L2[c]) for c in range(o.dim)]
            dW = [dW[c] / 3.0 + (2.0 / 3.0) * (dS2[c] + k * dL2[c]) for c in range(o.dim)]
        return dW

    def rk3_vjp(self, V, lam):
        o = self.o
        k = o.dt / o.nsub
        states, _ = self._rk3_states(V)
        for W, S1, S2 in reversed(states):
            t = self.convection_vjp(S2, lam)
            lS2 = [(2.0 / 3.0) * (lam[c] + k * t[c]) for c in range(o.dim)]
            lW = [lam[c] / 3.0 for c in range(o.dim)]
            t = self.convection_vjp(S1, lS2)
            lS1 = [0.25 * (lS2[c] + k * t[c]) for c in range(o.dim)]
            lW = [lW[c] + 0.75 * lS2[c] for c in range(o.dim)]
            t = self.convection_vjp(W, lS1)
            lam = [lW[c] + lS1[c] + k * t[c] for c in range(o.dim)]
        return lam

    # ----------------------------------------------------------------- one step
    def _forward(self, Us, P):
        o = self.o
        V = [o.dual_to_main(Us[d], d) for d in range(o.dim)]
        F = o.rk3(V)
        Vh = [o.viscous_solve_exact(o.mass_all(F[c])) for c in range(o.dim)]
        Ustar = [o.main_to_dual(Vh[d], d) for d in range(o.dim)]
        return V, F, Vh, Ustar

    def step_jvp(self, Us, P, dUs, dP, dnu=0.0):
        """(dU_new, dP_new) of step_exact at (Us, P, nu) in the direction
        (dUs, dP, dnu)."""
        o = self.o
        V, F, Vh, Ustar = self._forward(Us, P)
        dV = [o.dual_to_main(dUs[d], d) for d in range(o.dim)]
        dF = self.rk3_jvp(V, dV)
        # (M + nu A') Vh = M F  =>  (M + nu A') dVh = M dF - dnu A' Vh
        dVh = [o.viscous_solve_exact(o.mass_all(dF[c]) - dnu * o.Aprime(Vh[c])) for c in range(o.dim)]
        dUstar = [o.main_to_dual(dVh[d], d) for d in range(o.dim)]
        db = o.pressure_rhs(dUstar, dP)
        db = db - np.mean(db)
        dx = o.pressure_solve_exact(db, dP)  # A^+ db + K(dP)
        dPn = dx - o.physical_mean(dx)
        dq = o.theta * dPn + (1.0 - o.theta) * dP
        return o.velocity_update(dUstar, dq), dPn

    def step_vjp(self, Us, P, lamU, lamP):
        """Adjoint of step_exact at (Us, P, nu): given the cotangents of
        (U_new, P_new), return those of (Us, P) and d/dnu."""
        o = self.o
        V, F, Vh, Ustar = self._forward(Us, P)
        # velocity update
        lUstar = [u.copy() for u in lamU]
        lq = np.zeros(o.shape)
        for d in range(o.dim):
            lq -= (o.dt / o.g.dx[d]) * self.weak_gradient_T(o.along(o.B.Minv, lamU[d], d), d)
        lPn = lamP + o.theta * lq
        lP = (1.0 - o.theta) * lq
        # gauge; the pressure solve is x = (I - K) G b + K(P) with G the
        # symmetric spectral inverse and K the Euclidean kernel projection,
        # so lam_b = G (I - K) lam_x and the kernel part of lam_x goes to P
        lx = self.gauge_T(lPn)
        kx = o.kernel_part(lx)
        lP = lP + kx
        lb = o.block_circulant_solve(lx - kx, None, 0.0, o.theta, raw=True)
        lb = lb - np.mean(lb)
        # b = -div U* - (1 - theta) A' P
        dT = self.divergence_T(lb)
        lUstar = [lUstar[d] - dT[d] for d in range(o.dim)]
        lP = lP - (1.0 - o.theta) * o.Aprime(lb)
        # projections back, viscous solve (symmetric) and its nu-derivative
        lVh = [self.main_to_dual_T(lUstar[d], d) for d in range(o.dim)]
        mu = [o.viscous_solve_exact(lVh[c]) for c in range(o.dim)]
        dnu = -sum(float(np.sum(mu[c] * o.Aprime(Vh[c]))) for c in range(o.dim))
        lF = [o.mass_all(mu[c]) for c in range(o.dim)]
        lV = self.rk3_vjp(V, lF)
        lU = [self.dual_to_main_T(lV[d], d) for d in range(o.dim)]
        return lU, lP, dnu
