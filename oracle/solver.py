"""One load increment of the FFT-Galerkin SGCP problem (oracle; test
infrastructure only).

Per increment k (Sec. 2.2 with the readings listed in the package doc):
 1. Nye tensor G = -curl Fp_{k-1} by the rotated stencil (App. B, App. A).
 2. GND densities: rho18 = A^T (A A^T)^{-1} vec G (Eq. mingnd, read as the
    minimum-norm solution), A in the grain's sample frame (Eq. defA2); per slip
    system rho_GND^a = |rho_edge^a| + 1/2 |rho_screw^{d(a)}| (each <110> screw
    direction is shared by the two systems that glide along it; the paper does
    not say how the 18 segment densities map onto the 12 systems).
 3. Hardening, frozen over the increment:
      tauc^a = tau0 + alpha mu b sqrt(sum_b q^ab (rho_SSD^b + rho_GND^b))
    (Eq. Taylor_hard with the lattice friction tau0 and Taylor coefficient
    alpha of the workload; q normalised by its self term), and the mean free
    path l^a = K / sqrt(sum_{b != a} (rho_SSD^b + rho_GND^b)) (Eq. meanfree).
 4. Newton-Raphson on G*(P(F) - Pbar) = 0 (Eqs. eql_discrete2, linequil2ast):
    start F = F_{k-1} + dFbar on the strain-controlled components; each
    iteration evaluates the local update at every voxel, the residual
    R = G*(P - Pbar), and solves G*(K : dF) = -R by conjugate gradients
    from dF = 0.  Stop when rms(R) <= newton_tol * max(|<P>|, 1e-4 mu) (the
    paper stops on the size of dF; the residual test is the stricter reading).
    The Newton step is damped by halving until rms(R) (absolute) decreases.
 5. Commit: Kocks-Mecking (Eq. kocks) integrated implicitly over the increment,
      rho_SSD <- (rho_SSD + |dgam|/(b l)) / (1 + 2 y_c |dgam| / b),
    then Fp, S and F.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import crystal as cr
from . import constitutive as co
from . import spectral as sp


@dataclass
class Options:
    newton_tol: float = 1e-11
    cg_tol: float = 1e-11
    local_tol: float = 1e-14
    max_newton: int = 40
    max_cg: int = 2000
    max_halvings: int = 12
    extrapolate: bool = True


@dataclass
class StepInfo:
    newton_iters: int = 0
    cg_iters: list = field(default_factory=list)
    residuals: list = field(default_factory=list)
    dF_inf: list = field(default_factory=list)
    local_max_iters: int = 0
    local_failures: int = 0
    converged: bool = False
    seconds: float = 0.0


class RVE:
    """Voxelised polycrystal state.  grain_id has numpy shape (n2, n1, n0)."""

    def __init__(self, grain_id, quat, mat, L, opts: Options | None = None):
        self.gid = np.asarray(grain_id, dtype=np.int64)
        self.shape = self.gid.shape
        self.h = L / self.shape[2]
        self.mat = mat
        self.opts = opts or Options()
        self.mu = mat.mu if mat.mu > 0 else cr.shear_modulus(mat.C11, mat.C12, mat.C44)
        self.q = cr.interaction_matrix(mat.q, mat.q_normalise)
        self.screw = cr.screw_of_system()
        s, m = cr.slip_systems()
        Cc = cr.cubic_stiffness(mat.C11, mat.C12, mat.C44)
        self.grains = []
        for g in range(len(quat)):
            idx = np.nonzero(self.gid.ravel() == g)[0]
            if len(idx) == 0:
                continue
            R = cr.rotation(quat[g])
            self.grains.append(dict(
                idx=idx, R=R, C=cr.rotate4(Cc, R),
                S0=np.einsum("ai,aj->aij", s @ R.T, m @ R.T),
                A=cr.nye_matrix(R, mat.b)))
        nv = self.gid.size
        self.F = np.tile(np.eye(3), (nv, 1, 1))
        self.Fp = np.tile(np.eye(3), (nv, 1, 1))
        self.S = np.zeros((nv, 3, 3))
        self.rho_ssd = np.full((nv, 12), mat.rho0_total / 12.0)
        self.rho_gnd = np.zeros((nv, 12))
        self.rho18 = np.zeros((nv, 18))
        self.G = np.zeros((nv, 3, 3))
        self.P = np.zeros((nv, 3, 3))
        self.Fbar = np.eye(3)
        self.t = 0.0
        self.increment = 0

    # -- helpers ------------------------------------------------------------
    def field(self, flat):
        """(nv, ...) -> (n2, n1, n0, ...)."""
        return flat.reshape(self.shape + flat.shape[1:])

    def flat(self, fld):
        return fld.reshape((-1,) + fld.shape[3:])

    def hardening(self):
        """Steps 1-3: Nye tensor, GND densities, tauc and mean free path."""
        m = self.mat
        G = self.flat(sp.nye_tensor(self.field(self.Fp), self.h))
        rho18 = np.zeros((G.shape[0], 18))
        for gr in self.grains:
            rho18[gr["idx"]] = cr.min_norm_gnd(gr["A"], G[gr["idx"]].reshape(-1, 9).T).T
        rho_gnd = np.abs(rho18[:, :12]) + 0.5 * np.abs(rho18[:, 12 + self.screw])
        if not m.gnd_enabled:
            rho_gnd = np.zeros_like(rho_gnd)
        rho = self.rho_ssd + rho_gnd
        tauc = m.tau0 + m.alpha * self.mu * m.b * np.sqrt(rho @ self.q.T)
        ell = m.K / np.sqrt(rho.sum(axis=1, keepdims=True) - rho)
        self.G, self.rho18, self.rho_gnd = G, rho18, rho_gnd
        return tauc, ell

    def constitutive(self, F, tauc, S_init, dt, tangent=True):
        nv = F.shape[0]
        P = np.empty((nv, 3, 3)); S = np.empty((nv, 3, 3)); M = np.empty((nv, 3, 3))
        dg = np.empty((nv, 12)); K = np.empty((nv, 3, 3, 3, 3)) if tangent else None
        it_max, fails = 0, 0
        for gr in self.grains:
            i = gr["idx"]
            r = co.local_update(F[i], self.Fp[i], tauc[i], S_init[i], gr["C"], gr["S0"], dt,
                                self.mat.gdot0, self.mat.n, self.opts.local_tol * self.mu,
                                tangent=tangent)
            P[i], S[i], M[i], dg[i] = r.P, r.S, r.M, r.dgam
            if tangent:
                K[i] = r.K
            it_max = max(it_max, int(r.iters.max(initial=0)))
            fails += int(r.failed.sum())
        return P, K, S, M, dg, it_max, fails

    def stress_scale(self, P):
        return max(float(np.linalg.norm(P.mean(axis=0))), 1e-4 * self.mu)

    def rms(self, X):
        return float(np.sqrt(np.mean(np.sum(X.reshape(X.shape[0], -1) ** 2, axis=1))))

    # -- one increment ------------------------------------------------------
    def step(self, dFbar, strain_mask, Pbar, dt):
        t0 = time.perf_counter()
        o = self.opts
        mask = np.asarray(strain_mask, dtype=np.uint8).reshape(9)
        info = StepInfo()
        tauc, ell = self.hardening()
        dFb = (np.asarray(dFbar).reshape(9) * mask).reshape(3, 3)
        if o.extrapolate and self.increment > 0:
            # predictor: extrapolate the last increment's change of F (its
            # fluctuation is compatible) and reset the strain-controlled means;
            # the converged answer does not depend on the starting point
            d = (self.F - self.F_prev) * (dt / self.dt_prev)
            d = d - d.mean(axis=0) * mask.reshape(3, 3)
            F = self.F + d + dFb
        else:
            F = self.F + dFb
        Pbar_f = (np.asarray(Pbar).reshape(9) * (1 - mask)).reshape(3, 3)
        S_it = self.S.copy()
        P, K, S_it, M, dg, lit, lf = self.constitutive(F, tauc, S_it, dt)
        info.local_max_iters, info.local_failures = lit, lf
        R = self.flat(sp.project(self.field(P - Pbar_f), mask, self.h))
        rabs = self.rms(R)
        res = rabs / self.stress_scale(P)
        info.residuals.append(res)
        while lf == 0:
            if res <= o.newton_tol:
                info.converged = True
                break
            if info.newton_iters == o.max_newton:
                break
            dF, ncg = self.cg(K, -R, mask)
            info.cg_iters.append(ncg)
            # backtracking on the residual norm (the paper gives no globalisation
            # of its Newton-Raphson; halving the step leaves the solution unchanged)
            lam = 1.0
            for _ in range(o.max_halvings + 1):
                trial = self.constitutive(F + lam * dF, tauc, S_it, dt)
                Rt = self.flat(sp.project(self.field(trial[0] - Pbar_f), mask, self.h))
                rt = self.rms(Rt)
                if trial[6] == 0 and rt < rabs:
                    break
                lam *= 0.5
            P, K, S_it, M, dg, lit, lf = trial
            info.local_max_iters = max(info.local_max_iters, lit)
            info.local_failures += lf
            F = F + lam * dF
            R, rabs = Rt, rt
            res = rabs / self.stress_scale(P)
            info.residuals.append(res)
            info.dF_inf.append(float(lam * np.abs(dF).max()))
            info.newton_iters += 1
        info.seconds = time.perf_counter() - t0
        if not info.converged:
            return info
        m = self.mat
        adg = np.abs(dg)
        self.rho_ssd = (self.rho_ssd + adg / (m.b * ell)) / (1.0 + 2.0 * m.yc * adg / m.b)
        self.Fp = M @ self.Fp
        self.F_prev, self.dt_prev = self.F, dt
        self.S, self.F, self.P = S_it, F, P
        self.Fbar = F.mean(axis=0)
        self.t += dt
        self.increment += 1
        return info

    def cg(self, K, b, mask):
        """Conjugate gradients for G*(K : x) = b from x = 0 (b in the range of G*)."""
        o = self.opts
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        stop = (o.cg_tol ** 2) * rr
        for k in range(o.max_cg):
            if rr <= stop:
                return x, k
            q = self.flat(sp.project(self.field(np.einsum("vijkl,vkl->vij", K, p)), mask, self.h))
            alpha = rr / float(np.sum(p * q))
            x += alpha * p
            r -= alpha * q
            rr_new = float(np.sum(r * r))
            p = r + (rr_new / rr) * p
            rr = rr_new
        return x, o.max_cg

    # -- outputs --------------------------------------------------------------
    def macro_stress(self):
        P = self.P.mean(axis=0)
        J = np.linalg.det(self.F)
        sig = (self.P @ np.swapaxes(self.F, 1, 2)) / J[:, None, None]
        return P, sig.mean(axis=0)
