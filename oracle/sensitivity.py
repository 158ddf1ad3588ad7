"""Sensitivities of the macroscopic stress-strain curve with respect to the
material parameters theta = (tau0, K, alpha, b) (oracle; test infrastructure
only).

Forward mode through the same discrete equations the oracle solves per
increment k (Sec. 2.1, Sec. 2.2 and the readings in `solver.py`):

  hardening   rho18 = A(b)^+ G(Fp_{k-1}),  A proportional to b (Eq. defA2), so
              d rho18 = A^+ G(dFp_{k-1}) - rho18 db / b;
              rho_GND^a = |rho18_edge^a| + 1/2 |rho18_screw^d(a)|;
              tauc^a = tau0 + alpha mu b sqrt(sum_b q^ab rho^b) (Eq. Taylor_hard),
              l^a = K / sqrt(sum_{b != a} rho^b) (Eq. meanfree),
              rho = rho_SSD,k-1 + rho_GND;
  local       r(S; F, Fp_{k-1}, tauc) = 0 (backward Euler, implicit in S), so
              J dS = C : sym(Fe^T dFe|_S) with the change of Fe at fixed S;
              dgam = dt gdot0 |tau/tauc|^n sgn tau gives
              d dgam = dgam'(tau) (S0 : dS) - n dgam dtauc / tauc;
              Fp_k = M Fp_{k-1}, P = F Fp^-1 S Fp^-T (Eq. Piola);
  equilibrium G*(K : dF) = -G*(dP|_dF=0) (Eq. linequil2ast with the increment's
              consistent tangent K), with zero strain-controlled means of dF
              and zero stress-controlled means of dP (the loads do not depend
              on theta);
  commit      rho_SSD,k = (rho_SSD,k-1 + |dgam|/(b l)) / (1 + 2 y_c |dgam| / b)
              (Eq. kocks, integrated implicitly).

The state tangents d Fp_k and d rho_SSD,k carry the history to the next
increment.  A linear solve per parameter and increment, with the tangent of
the converged increment: no reverse sweep or checkpoints are needed for four
parameters.  Pinned against central finite differences of the oracle's own
curve (tests/test_oracle_sensitivity.py).
"""
from __future__ import annotations

import numpy as np

from . import constitutive as co
from . import crystal as cr
from . import spectral as sp

PARAMS = ("tau0", "K", "alpha", "b")


def _sym(X):
    return 0.5 * (X + np.swapaxes(X, -1, -2))


def _t(X):
    return np.swapaxes(X, -1, -2)


def local_jvp(F, Fp0, tauc, S, C, S0, dt, gdot0, n, dF, dFp0, dtauc):
    """Directional derivative of the converged local update at V voxels of one
    grain along (dF, dFp0, dtauc): returns dS, d dgam, dFp, dP."""
    Fp0inv = np.linalg.inv(Fp0)
    FeTr = F @ Fp0inv
    A = _t(FeTr) @ FeTr
    tau, dg, M, Minv, Ce, _ = co._evaluate(S, A, C, S0, tauc, dt, gdot0, n)
    w = co.tau_gradient(S0)
    J, dgp = co._jacobian(tau, Minv, Ce, C, S0, w, tauc, dt, gdot0, n)
    Fpinv = Fp0inv @ Minv
    Fe = F @ Fpinv
    dFp0inv = -Fp0inv @ dFp0 @ Fp0inv
    ddg_tc = -n * dg / tauc * dtauc                       # at fixed tau
    dMinv_tc = -Minv @ np.einsum("va,aij->vij", ddg_tc, S0) @ Minv
    dFe = dF @ Fpinv + F @ dFp0inv @ Minv + FeTr @ dMinv_tc
    rhs = co.to_voigt(np.einsum("ijkl,vkl->vij", C, _sym(_t(Fe) @ dFe)))
    dS = co.from_voigt(np.linalg.solve(J, rhs[..., None])[..., 0])
    ddg = dgp * np.einsum("vij,aij->va", dS, S0) + ddg_tc
    dM = np.einsum("va,aij->vij", ddg, S0)
    dMinv = -Minv @ dM @ Minv
    dFpinv = dFp0inv @ Minv + Fp0inv @ dMinv
    Q = Fpinv @ S @ _t(Fpinv)
    dQ = dFpinv @ S @ _t(Fpinv) + Fpinv @ dS @ _t(Fpinv) + Fpinv @ S @ _t(dFpinv)
    dP = dF @ Q + F @ dQ
    dFp = dM @ Fp0 + M @ dFp0
    return dS, ddg, dFp, dP


def hardening_jvp(rve, Fp_prev, rho_prev, dFp_prev, drho_prev, dtheta):
    """tauc, l and their derivatives along (dFp_prev, drho_prev, dtheta) from
    the state at the start of the increment."""
    m = rve.mat
    dtau0, dK, dalpha, db = dtheta
    G = rve.flat(sp.nye_tensor(rve.field(Fp_prev), rve.h))
    dG = rve.flat(sp.nye_tensor(rve.field(dFp_prev), rve.h))
    nv = G.shape[0]
    rho18, drho18 = np.zeros((nv, 18)), np.zeros((nv, 18))
    for gr in rve.grains:
        i = gr["idx"]
        rho18[i] = cr.min_norm_gnd(gr["A"], G[i].reshape(-1, 9).T).T
        drho18[i] = cr.min_norm_gnd(gr["A"], dG[i].reshape(-1, 9).T).T
    drho18 = drho18 - rho18 * (db / m.b)
    scr = 12 + rve.screw
    if m.gnd_enabled:
        rho_gnd = np.abs(rho18[:, :12]) + 0.5 * np.abs(rho18[:, scr])
        drho_gnd = np.sign(rho18[:, :12]) * drho18[:, :12] + 0.5 * np.sign(rho18[:, scr]) * drho18[:, scr]
    else:
        rho_gnd = drho_gnd = np.zeros((nv, 12))
    rho, drho = rho_prev + rho_gnd, drho_prev + drho_gnd
    X = np.sqrt(rho @ rve.q.T)
    dX = (drho @ rve.q.T) / (2.0 * X)
    tauc = m.tau0 + m.alpha * rve.mu * m.b * X
    dtauc = dtau0 + rve.mu * (dalpha * m.b * X + m.alpha * db * X + m.alpha * m.b * dX)
    Y = np.sqrt(rho.sum(axis=1, keepdims=True) - rho)
    dY = (drho.sum(axis=1, keepdims=True) - drho) / (2.0 * Y)
    ell = m.K / Y
    dell = dK / Y - m.K * dY / Y ** 2
    return tauc, dtauc, ell, dell


def commit_jvp(rho_prev, drho_prev, dg, ddg, ell, dell, b, db, yc):
    a = np.abs(dg)
    da = np.sign(dg) * ddg
    num = rho_prev + a / (b * ell)
    dnum = drho_prev + da / (b * ell) - a * (db * ell + b * dell) / (b * ell) ** 2
    D = 1.0 + 2.0 * yc * a / b
    dD = 2.0 * yc * (da / b - a * db / b ** 2)
    rho = num / D
    return rho, (dnum - rho * dD) / D


class SensitivityRVE:
    """An oracle RVE that also carries d Fp and d rho_SSD for each parameter of
    PARAMS; step() returns the increment's info and d<P>/d theta (4, 3, 3)."""

    def __init__(self, rve):
        self.rve = rve
        nv = rve.gid.size
        self.dFp = np.zeros((len(PARAMS), nv, 3, 3))
        self.drho = np.zeros((len(PARAMS), nv, 12))

    def step(self, dFbar, strain_mask, Pbar, dt):
        r = self.rve
        m = r.mat
        mask = np.asarray(strain_mask, dtype=np.uint8).reshape(9)
        Fp_prev, rho_prev = r.Fp.copy(), r.rho_ssd.copy()
        info = r.step(dFbar, strain_mask, Pbar, dt)
        if not info.converged:
            return info, None
        F, S = r.F, r.S
        nv = F.shape[0]
        dPbar = np.zeros((len(PARAMS), 3, 3))
        for j in range(len(PARAMS)):
            dtheta = np.zeros(4)
            dtheta[j] = 1.0
            tauc, dtauc, ell, dell = hardening_jvp(r, Fp_prev, rho_prev, self.dFp[j], self.drho[j], dtheta)
            K = np.empty((nv, 3, 3, 3, 3))
            dPq = np.empty((nv, 3, 3))
            for gr in r.grains:
                i = gr["idx"]
                lr = co.local_update(F[i], Fp_prev[i], tauc[i], S[i], gr["C"], gr["S0"], dt, m.gdot0, m.n,
                                     r.opts.local_tol * r.mu, tangent=True)
                K[i] = lr.K
                dPq[i] = local_jvp(F[i], Fp_prev[i], tauc[i], S[i], gr["C"], gr["S0"], dt, m.gdot0, m.n,
                                   np.zeros_like(F[i]), self.dFp[j][i], dtauc[i])[3]
            b = -r.flat(sp.project(r.field(dPq), mask, r.h))
            dF, _ = r.cg(K, b, mask)
            dP = np.empty((nv, 3, 3))
            dFp = np.empty((nv, 3, 3))
            ddg = np.empty((nv, 12))
            dg = np.empty((nv, 12))
            for gr in r.grains:
                i = gr["idx"]
                _, ddg[i], dFp[i], dP[i] = local_jvp(F[i], Fp_prev[i], tauc[i], S[i], gr["C"], gr["S0"], dt,
                                                     m.gdot0, m.n, dF[i], self.dFp[j][i], dtauc[i])
                Fp0inv = np.linalg.inv(Fp_prev[i])
                FeTr = F[i] @ Fp0inv
                dg[i] = co._evaluate(S[i], _t(FeTr) @ FeTr, gr["C"], gr["S0"], tauc[i], dt, m.gdot0, m.n)[1]
            _, self.drho[j] = commit_jvp(rho_prev, self.drho[j], dg, ddg, ell, dell, m.b, dtheta[3], m.yc)
            self.dFp[j] = dFp
            dPbar[j] = dP.mean(axis=0)
        return info, dPbar
