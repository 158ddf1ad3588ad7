"""Physics pins of the oracle's constitutive update and incremental solver
(Sec. 2.1-2.2): elastic limit, objectivity, consistent tangent vs finite
differences, homogeneous RVE vs an independent point solve, the exact
two-phase laminate, Voigt/Reuss bounds, the Schmid-law flow stress of a
single crystal and the macroscopic invariants of the mixed control."""
import numpy as np
import pytest
import scipy.optimize as so

import rvegen
from oracle import constitutive as co
from oracle import crystal as cr
from oracle import solver
from oracle import spectral as sp

MASK = rvegen.UNIAXIAL_X_MASK
VP6 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def grain_tables(mat, quat):
    R = cr.rotation(quat)
    s, m = cr.slip_systems()
    C = cr.rotate4(cr.cubic_stiffness(mat.C11, mat.C12, mat.C44), R)
    return C, np.einsum("ai,aj->aij", s @ R.T, m @ R.T)


def svk_P(F, C):
    """St-Venant-Kirchhoff: P = F (C : E), E = (F^T F - I)/2 (textbook)."""
    E = 0.5 * (F.T @ F - np.eye(3))
    return F @ np.einsum("ijkl,kl->ij", C, E)


def voigt66(C):
    return np.array([[C[i, j, k, l] for (k, l) in VP6] for (i, j) in VP6])


def test_local_update_elastic_limit_is_svk():
    mat = rvegen.material("Cu")
    C, S0 = grain_tables(mat, rvegen.random_quaternions(1, 11)[0])
    rng = np.random.default_rng(0)
    F = np.eye(3) + 3e-3 * rng.standard_normal((6, 3, 3))
    r = co.local_update(F, np.tile(np.eye(3), (6, 1, 1)), np.full((6, 12), 1e9), np.zeros((6, 3, 3)),
                        C, S0, 1.0, 1e-3, 20.0, 1e-10)
    for v in range(6):
        assert np.allclose(r.P[v], svk_P(F[v], C), rtol=0, atol=1e-9)
    assert np.abs(r.dgam).max() < 1e-100


def test_local_update_objectivity():
    mat = rvegen.material("Cu")
    C, S0 = grain_tables(mat, rvegen.random_quaternions(1, 12)[0])
    rng = np.random.default_rng(1)
    F = np.eye(3) + 2e-3 * rng.standard_normal((4, 3, 3))
    Fp0 = np.eye(3) + 1e-3 * rng.standard_normal((4, 3, 3))
    Q = cr.rotation(rvegen.random_quaternions(1, 13)[0])
    args = (np.full((4, 12), 12.0), np.zeros((4, 3, 3)), C, S0, 1.0, 1e-3, 20.0, 3e-10)
    a = co.local_update(F, Fp0, *args)
    b = co.local_update(Q @ F, Fp0, *args)
    assert np.abs(a.dgam).max() > 1e-4                        # plastic
    assert np.allclose(b.S, a.S, atol=1e-9)
    assert np.allclose(b.P, Q @ a.P, atol=1e-9)
    assert np.allclose(b.K, np.einsum("ia,vajkl,kb->vijbl", Q, a.K, Q.T), atol=1e-5)


def test_consistent_tangent_matches_central_differences():
    mat = rvegen.material("Cu")
    C, S0 = grain_tables(mat, rvegen.random_quaternions(1, 5)[0])
    rng = np.random.default_rng(1)
    F = np.eye(3) + 2e-3 * rng.standard_normal((4, 3, 3))
    Fp0 = np.eye(3) + 1e-3 * rng.standard_normal((4, 3, 3))
    tauc = np.full((4, 12), 12.7)
    mu = cr.shear_modulus(mat.C11, mat.C12, mat.C44)
    r = co.local_update(F, Fp0, tauc, np.zeros((4, 3, 3)), C, S0, 1.0, 1e-3, 20.0, 1e-14 * mu)
    assert np.abs(r.dgam).max() > 1e-3
    h = 1e-7
    Kfd = np.empty_like(r.K)
    for k in range(3):
        for l in range(3):
            d = np.zeros((3, 3)); d[k, l] = h
            rp = co.local_update(F + d, Fp0, tauc, r.S, C, S0, 1.0, 1e-3, 20.0, 1e-14 * mu, tangent=False)
            rm = co.local_update(F - d, Fp0, tauc, r.S, C, S0, 1.0, 1e-3, 20.0, 1e-14 * mu, tangent=False)
            Kfd[..., k, l] = (rp.P - rm.P) / (2 * h)
    assert np.abs(Kfd - r.K).max() < 1e-6 * np.abs(r.K).max()


def point_solve(mat, quat, Fbar_strain, state, dt, Pbar=np.zeros(9)):
    """Homogeneous mixed-control problem without any projection: find the five
    stress-controlled components of F with P_IJ(F) = Pbar_IJ (scipy root)."""
    C, S0 = grain_tables(mat, quat)
    mu = cr.shear_modulus(mat.C11, mat.C12, mat.C44)
    free = np.nonzero(MASK == 0)[0]
    Fp0, tauc, S_init = state

    def P_of(xf):
        F = Fbar_strain.copy().reshape(9); F[free] = xf
        r = co.local_update(F.reshape(1, 3, 3), Fp0[None], tauc[None], S_init[None], C, S0, dt,
                            mat.gdot0, mat.n, 1e-14 * mu, tangent=False)
        return r
    x0 = Fbar_strain.reshape(9)[free]
    sol = so.root(lambda xf: (P_of(xf).P.reshape(9)[free] - Pbar[free]) / mu, x0, method="hybr",
                  options=dict(xtol=1e-15))
    r = P_of(sol.x)
    F = Fbar_strain.copy().reshape(9); F[free] = sol.x
    return F.reshape(3, 3), r


@pytest.mark.parametrize("n", [1, 3, 4])
def test_homogeneous_rve_matches_point_solve(n):
    mat = rvegen.material("Cu")
    quat = rvegen.random_quaternions(1, 21)
    gid = np.zeros((n, n, n), dtype=np.int32)
    rve = solver.RVE(gid, quat, mat, 10e-6)
    dt, dFb = 1.0, np.array([1e-3, 0, 0, 0, 0, 0, 0, 0, 0])
    Fbar = np.eye(3)
    state = (np.eye(3), None, np.zeros((3, 3)))
    for k in range(3):
        tauc, _ = rve.hardening()
        state = (rve.Fp[0].copy(), tauc[0].copy(), rve.S[0].copy())
        info = rve.step(dFb, MASK, np.zeros(9), dt)
        assert info.converged
        Fbar = Fbar + dFb.reshape(3, 3)
        Fp, r = point_solve(mat, quat[0], np.where(MASK.reshape(3, 3) == 1, Fbar, np.eye(3) * 0 + Fbar), state, dt)
        assert np.abs(rve.F - rve.F[0]).max() < 1e-12                   # uniform
        assert np.abs(rve.P - rve.P[0]).max() < 1e-9
        assert np.allclose(rve.F[0], Fp, rtol=0, atol=1e-12)
        assert np.allclose(rve.P[0], r.P[0], rtol=0, atol=1e-8)
    assert np.abs(rve.Fp[0] - np.eye(3)).max() > 1e-4                   # it did yield
    assert np.abs(rve.G).max() == 0.0                                    # no GND in a uniform field


def test_elastic_laminate_exact_solution():
    mat = rvegen.material("Cu", tau0=1e9)
    quat = rvegen.random_quaternions(2, 31)
    n = 4
    gid = np.zeros((n, n, n), dtype=np.int32); gid[n // 2:] = 1        # layers normal to z
    rve = solver.RVE(gid, quat, mat, 10e-6)
    dFb = np.array([1e-3, 0, 0, 0, 0, 0, 0, 0, 0])
    info = rve.step(dFb, MASK, np.zeros(9), 1.0)
    assert info.converged
    # exact: F^A - F^B = a (x) e_z, (F^A + F^B)/2 has the prescribed strain parts,
    # traction P e_z continuous, the stress-controlled mean of P vanishes
    CA, _ = grain_tables(mat, quat[0]); CB, _ = grain_tables(mat, quat[1])
    free = np.nonzero(MASK == 0)[0]

    def unpack(x):
        Fm = np.eye(3).reshape(9) + dFb; Fm[free] = Fm[free] + x[3:]
        Fm = Fm.reshape(3, 3)
        J = np.outer(x[:3], [0, 0, 1.0])
        return Fm + 0.5 * J, Fm - 0.5 * J

    def eqs(x):
        FA, FB = unpack(x)
        PA, PB = svk_P(FA, CA), svk_P(FB, CB)
        return np.concatenate([(PA - PB)[:, 2], (0.5 * (PA + PB)).reshape(9)[free]]) / 1e5
    sol = so.root(eqs, np.zeros(8), method="hybr", options=dict(xtol=1e-15))
    FA, FB = unpack(sol.x)
    Fz = rve.field(rve.F)
    assert np.allclose(Fz[: n // 2], FA, rtol=0, atol=1e-12)
    assert np.allclose(Fz[n // 2:], FB, rtol=0, atol=1e-12)
    assert np.abs(sol.x[:3]).max() > 1e-5                               # a real jump


def test_voigt_reuss_bounds_elastic_polycrystal():
    mat = rvegen.material("Cu", tau0=1e9)
    gid, _ = rvegen.voronoi_grain_map(8, 8, 41)
    quat = rvegen.random_quaternions(8, 42)
    rve = solver.RVE(gid, quat, mat, 10e-6)
    eps = 1e-5
    info = rve.step(np.array([eps, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), 1.0)
    assert info.converged
    P, _ = rve.macro_stress()
    E_app = P[0, 0] / eps
    Cv = np.zeros((gid.size, 6, 6))
    for gr in rve.grains:
        Cv[gr["idx"]] = voigt66(gr["C"])
    E_voigt = 1.0 / np.linalg.inv(Cv.mean(axis=0))[0, 0]
    E_reuss = 1.0 / np.linalg.inv(Cv).mean(axis=0)[0, 0]
    assert E_reuss * (1 - 1e-4) < E_app < E_voigt * (1 + 1e-4)
    assert E_voigt - E_reuss > 0.1 * E_reuss                             # the bounds are apart


def test_schmid_law_flow_stress_single_crystal():
    # [100] tension of a cube-oriented crystal: 8 systems with Schmid factor
    # 1/sqrt(6) share the plastic stretching rate equally, so at steady state
    # gdot = eps_true_rate / (8 m) and sigma = (tau0 / m) (gdot / gdot0)^(1/n).
    mat = rvegen.material("Cu", alpha=0.0, gnd_enabled=False)
    rve = solver.RVE(np.zeros((1, 1, 1), dtype=np.int32), np.array([[1.0, 0, 0, 0]]), mat, 10e-6)
    rate, dt, n_inc = 1e-3, 1.0, 20
    for k in range(n_inc):
        info = rve.step(np.array([rate * dt, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), dt)
        assert info.converged
    _, sig = rve.macro_stress()
    m = 1.0 / np.sqrt(6.0)
    eps = rate * dt * n_inc
    expected = (mat.tau0 / m) * (rate / (1 + eps) / (8 * m * mat.gdot0)) ** (1.0 / mat.n)
    assert abs(sig[0, 0] / expected - 1) < 1e-3, (sig[0, 0], expected)
    assert abs(sig[1, 1]) < 1e-9 and abs(sig[2, 2]) < 1e-9


def test_macro_invariants_after_plastic_increments():
    wl = rvegen.Workload("t", 8, 6, "Cu", 0.002, 2, seed=77)
    gid, quat, mat = wl.inputs()
    rve = solver.RVE(gid, quat, mat, wl.edge)
    for k in range(2):
        info = rve.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert info.converged and info.local_failures == 0
    Fm = rve.F.mean(axis=0).reshape(9)
    assert np.allclose(Fm[MASK == 1], (np.eye(3).reshape(9) + 2 * wl.dFbar())[MASK == 1], atol=1e-15)
    Pm = rve.P.mean(axis=0).reshape(9)
    assert np.abs(Pm[MASK == 0]).max() < 1e-9 * np.abs(Pm).max()
    R = sp.project(rve.field(rve.P), MASK, rve.h)
    assert np.sqrt(np.mean(R ** 2)) < 1e-10 * np.abs(Pm).max()
    assert rve.rho_gnd.max() > 0 and np.abs(rve.Fp - np.eye(3)).max() > 1e-4
    # SSD densities only grow under Kocks-Mecking far below saturation
    assert (rve.rho_ssd >= mat.rho0_total / 12 - 1e-3).all()
