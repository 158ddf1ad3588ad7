"""Per-voxel crystal-plasticity update and consistent tangent (oracle; test
infrastructure only).

Sec. 2.1 of the paper, vectorised over the voxels of one grain:
  F = Fe Fp                                   (Eq. 1)
  Lp = sum_a gdot^a s^a (x) m^a               (Eq. 2)
  Ee = 1/2 (Fe^T Fe - I)                      (Eq. 3)
  S = C : Ee                                  (Eq. 4)
  tau^a = S : (s^a (x) m^a)                   (Eq. 5)
  gdot^a = gdot0 |tau^a / tauc^a|^n sgn tau^a  (power law; Table 1 gives the
           rate sensitivity m = 0.05, read as exponent n = 1/m = 20)
  P = Fe S Fe^T F^{-T}                        (Eq. Piola)

Time integration (the paper is silent; reading): backward Euler,
  Fp = (I + sum_a dgam^a s^a (x) m^a) Fp_prev,  dgam^a = dt gdot^a(tau^a(S)),
with tauc frozen over the increment.  The unknown is S (6 components); the
residual r(S) = S - C : Ee(S) is solved by Newton with the exact Jacobian and
step halving (accept a step only if |r| decreases and every |dgam| <= DGAM_MAX).
The consistent tangent K = dP/dF (named in Eq. linequil2ast, never derived in
the paper) is the implicit-function derivative through S(F) and Fp(S); it is
pinned against central finite differences of this same update.
"""
from __future__ import annotations

import numpy as np

VP = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
DGAM_MAX = 0.1
I3 = np.eye(3)


def to_voigt(X):
    return np.stack([X[..., i, j] for i, j in VP], axis=-1)


def from_voigt(v):
    X = np.empty(v.shape[:-1] + (3, 3))
    for a, (i, j) in enumerate(VP):
        X[..., i, j] = v[..., a]
        X[..., j, i] = v[..., a]
    return X


def tau_gradient(S0):
    """d tau / d S_voigt for tau = S : S0 with S symmetric: (12, 6)."""
    w = np.empty(S0.shape[:-2] + (6,))
    for a, (i, j) in enumerate(VP):
        w[..., a] = S0[..., i, j] if i == j else S0[..., i, j] + S0[..., j, i]
    return w


class LocalResult:
    pass


def _evaluate(S, A, C, S0, tauc, dt, gdot0, n):
    tau = np.einsum("vij,aij->va", S, S0)
    x = tau / tauc
    with np.errstate(over="ignore", invalid="ignore"):
        dg = dt * gdot0 * np.abs(x) ** n * np.sign(x)
    # a trial with |dgam| above DGAM_MAX is rejected by the caller; give it an
    # infinite residual without forming M (which could be singular)
    bad = ~np.all(np.isfinite(dg) & (np.abs(dg) <= DGAM_MAX), axis=-1)
    M = I3 + np.einsum("va,aij->vij", np.where(bad[:, None], 0.0, dg), S0)
    Minv = np.linalg.inv(M)
    Ce = np.swapaxes(Minv, 1, 2) @ A @ Minv
    Ee = 0.5 * (Ce - I3)
    Snew = np.einsum("ijkl,vkl->vij", C, Ee)
    r = to_voigt(S - Snew)
    r[bad] = np.inf
    return tau, dg, M, Minv, Ce, r


def _jacobian(tau, Minv, Ce, C, S0, w, tauc, dt, gdot0, n):
    x = tau / tauc
    dgp = dt * gdot0 * n * np.abs(x) ** (n - 1) / tauc            # d dgam / d tau
    T = np.einsum("vik,akl,vlj->vaij", Ce, S0, Minv)              # Ce S0^a M^-1
    symT = 0.5 * (T + np.swapaxes(T, 2, 3))
    c = -to_voigt(np.einsum("ijkl,vakl->vaij", C, symT)) * dgp[..., None]   # (v, a, 6)
    return np.eye(6) - np.einsum("vab,ac->vbc", c, w), dgp


def local_update(F, Fp0, tauc, S_init, C, S0, dt, gdot0, n, tol_abs, max_iter=60,
                 tangent=True, floor_abs=None):
    """Implicit update at V voxels of one grain.

    F, Fp0, S_init: (V, 3, 3); tauc: (V, 12); C: (3, 3, 3, 3) sample frame;
    S0: (12, 3, 3) = s^a (x) m^a, sample frame.  Converges max_a |r_a| <= tol_abs.
    Returns a LocalResult with S, P, K (V, 3, 3, 3, 3; K_ijkl = dP_ij/dF_kl),
    dgam, M (= Fp Fp_prev^-1), iteration counts and a failure mask.  A voxel
    whose |r| can no longer be decreased is accepted when |r| <= floor_abs
    (default 10 tol_abs): there the round-off of r itself has been reached.
    """
    V = F.shape[0]
    floor_abs = 10.0 * tol_abs if floor_abs is None else floor_abs
    w = tau_gradient(S0)
    Fp0inv = np.linalg.inv(Fp0)
    FeTr = F @ Fp0inv
    A = np.swapaxes(FeTr, 1, 2) @ FeTr
    S = S_init.copy()
    tau, dg, M, Minv, Ce, r = _evaluate(S, A, C, S0, tauc, dt, gdot0, n)
    rn = np.max(np.abs(r), axis=-1)
    iters = np.zeros(V, dtype=np.int64)
    active = rn > tol_abs
    for _ in range(max_iter):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        J, _ = _jacobian(tau[idx], Minv[idx], Ce[idx], C, S0, w, tauc[idx], dt, gdot0, n)
        step = -np.linalg.solve(J, r[idx][..., None])[..., 0]
        lam = np.ones(len(idx))
        pending = np.ones(len(idx), dtype=bool)
        for _h in range(40):
            p = np.nonzero(pending)[0]
            if len(p) == 0:
                break
            v = idx[p]
            St = S[v] + from_voigt(lam[p, None] * step[p])
            t_, dg_, M_, Mi_, Ce_, r_ = _evaluate(St, A[v], C, S0, tauc[v], dt, gdot0, n)
            rn_ = np.max(np.abs(r_), axis=-1)
            ok = np.isfinite(rn_) & (rn_ < rn[v]) & (np.max(np.abs(dg_), axis=-1) <= DGAM_MAX)
            acc = p[ok]
            va = idx[acc]
            S[va], tau[va], dg[va], M[va], Minv[va], Ce[va], r[va], rn[va] = (
                St[ok], t_[ok], dg_[ok], M_[ok], Mi_[ok], Ce_[ok], r_[ok], rn_[ok])
            pending[acc] = False
            lam[pending] *= 0.5
        iters[idx] += 1
        # no step decreased |r|: converged at the round-off floor if |r| is already
        # within floor_abs, otherwise a failure
        stalled = idx[pending]
        active = rn > tol_abs
        active[stalled] = False
        floor_ok = stalled[rn[stalled] <= floor_abs]
        rn[floor_ok] = 0.0
    res = LocalResult()
    res.failed = rn > tol_abs
    res.iters = iters
    res.S, res.dgam, res.M = S, dg, M
    Fpinv = Fp0inv @ Minv
    Fe = F @ Fpinv
    res.P = Fe @ S @ np.swapaxes(Fe, 1, 2) @ np.swapaxes(np.linalg.inv(F), 1, 2)
    res.Fp = M @ Fp0
    if not tangent:
        return res
    J, dgp = _jacobian(tau, Minv, Ce, C, S0, w, tauc, dt, gdot0, n)
    Q = Fpinv @ S @ np.swapaxes(Fpinv, 1, 2)
    K = np.empty((V, 3, 3, 3, 3))
    for k in range(3):
        for l in range(3):
            dF = np.zeros((3, 3)); dF[k, l] = 1.0
            dEe = np.swapaxes(Fe, 1, 2) @ dF @ Fpinv
            dEe = 0.5 * (dEe + np.swapaxes(dEe, 1, 2))
            rhs = to_voigt(np.einsum("ijkl,vkl->vij", C, dEe))
            dS = from_voigt(np.linalg.solve(J, rhs[..., None])[..., 0])
            ddg = dgp * np.einsum("vij,aij->va", dS, S0)
            dM = np.einsum("va,aij->vij", ddg, S0)
            dFpinv = -Fpinv @ dM @ Minv
            dQ = (dFpinv @ S @ np.swapaxes(Fpinv, 1, 2) + Fpinv @ dS @ np.swapaxes(Fpinv, 1, 2)
                  + Fpinv @ S @ np.swapaxes(dFpinv, 1, 2))
            K[:, :, :, k, l] = dF @ Q + F @ dQ
    res.K = K
    return res
