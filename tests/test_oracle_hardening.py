"""Pins of the oracle's hardening block (Sec. 2.1): the Taylor critical
resolved shear stress (Eq. Taylor_hard with the Table 1 coefficients), the
mean free path (Eq. meanfree), the implicit Kocks-Mecking SSD update
(Eq. kocks) and the map from the 18 minimum-norm GND segment densities
(Eq. mingnd) onto the 12 slip systems.

Each expected value below is derived by hand from the paper's formulas and
the FCC geometry, not by calling the oracle's own helpers:
  * a closed-form tauc and mean free path for equal SSD densities, from the
    row sum of Table 1 with its class counts 1/2/1/2/4/2 written out;
  * tauc for a density on one system only, with that system's interaction
    row (classes derived by hand from the slip geometry);
  * the Kocks-Mecking fixed point rho = 1/(2 y_c l), which the implicit
    update leaves unchanged for any slip increment, on a [100] crystal;
  * the saturated flow stress of that crystal from the closed-form tauc;
  * the SSD storage rate against an independent integration of
    d rho / d gamma = (1/l - 2 y_c rho) / b;
  * the 18 -> 12 map on a screw-character single-slip field, with the screw
    direction of each system written out as a table.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import rvegen
from oracle import crystal as cr
from oracle import solver

MASK = rvegen.UNIAXIAL_X_MASK
Q = dict(zip(("self", "coplanar", "collinear", "hirth", "glissile", "lomer"), rvegen.Q_TABLE1))

# Interaction classes of slip system 1 (plane (111), direction [-1 0 1])
# with systems 0..11, derived by hand: same plane -> coplanar; s.s' = -1 ->
# collinear (system 7, [1 0 -1]); s.s' = 0 -> Hirth (systems 4, 10); else the
# junction s -/+ s' lies in one of the two planes -> glissile, otherwise
# Lomer (systems 5: [0 1 1] in neither (111) nor (-111); 9: [-1 -1 0] in
# neither (111) nor (11-1)).
ROW1 = ("coplanar", "self", "coplanar", "glissile", "hirth", "lomer",
        "glissile", "collinear", "glissile", "lomer", "hirth", "glissile")

# Screw direction (index into [0 1 -1], [1 0 -1], [1 -1 0], [0 1 1], [1 0 1],
# [1 1 0]) parallel to the slip direction of each system.
SCREW_OF = (0, 1, 2, 0, 4, 5, 3, 1, 5, 3, 4, 2)

# [100] tension of a cube crystal: the four systems whose slip direction has
# no x component carry no resolved shear stress; the other eight slip
# equally with Schmid factor 1/sqrt(6).
INACTIVE = (0, 3, 6, 9)
ACTIVE = tuple(a for a in range(12) if a not in INACTIVE)


def cu_mu():
    # Table 2's formula for the <110>{111} shear modulus, Cu constants
    C11, C12, C44 = 168.4e3, 121.4e3, 75.4e3
    return 3.0 * C44 * (C11 - C12) / (4.0 * C44 + C11 - C12)


def one_voxel(mat, quat=(1.0, 0.0, 0.0, 0.0), n=1):
    return solver.RVE(np.zeros((n, n, n), dtype=np.int32), np.array([quat]), mat, 10e-6)


def test_taylor_tauc_and_mean_free_path_closed_form():
    # rho_SSD = 1e12 / 12 m^-2 on every system, no GND: every row of
    # q_hat = q / q_self sums the six Table 1 coefficients with their counts
    mat = rvegen.material("Cu", gnd_enabled=False)
    rve = one_voxel(mat, n=2)
    tauc, ell = rve.hardening()
    row_sum = (1 * 0.122 + 2 * 0.122 + 1 * 0.657 + 2 * 0.084 + 4 * 0.137 + 2 * 0.118) / 0.122  # 16.18852...
    rho = 1e12 / 12
    mu = cu_mu()                                                        # 30497.418 MPa
    tauc_exact = 10.0 + 0.3 * mu * 0.256e-9 * np.sqrt(row_sum * rho)    # 12.72043 MPa
    ell_exact = 6.0 / np.sqrt(11 * rho)                                 # 6.26680e-6 m
    assert abs(tauc_exact - 12.72043) < 1e-5
    assert np.abs(tauc / tauc_exact - 1).max() < 1e-13
    assert np.abs(ell / ell_exact - 1).max() < 1e-13


def test_taylor_interaction_row_of_a_single_system_density():
    # a small background density on every system plus a large one on
    # system 1: tauc^a = tau0 + alpha mu b sqrt(rowsum * bg + q_hat(a, 1) * big)
    mat = rvegen.material("Cu", gnd_enabled=False)
    rve = one_voxel(mat)
    bg, big = 1e9, 5e13
    rve.rho_ssd[:] = bg
    rve.rho_ssd[:, 1] += big
    tauc, ell = rve.hardening()
    row_sum = (Q["self"] + 2 * Q["coplanar"] + Q["collinear"] + 2 * Q["hirth"] + 4 * Q["glissile"]
               + 2 * Q["lomer"]) / Q["self"]
    mu = cu_mu()
    for a in range(12):
        qa1 = Q[ROW1[a]] / Q["self"]
        expect = 10.0 + 0.3 * mu * 0.256e-9 * np.sqrt(row_sum * bg + qa1 * big)
        assert abs(tauc[0, a] / expect - 1) < 1e-13, (a, ROW1[a])
        # the mean free path sums the other systems only (beta != alpha)
        others = 11 * bg + (big if a != 1 else 0.0)
        assert abs(ell[0, a] / (6.0 / np.sqrt(others)) - 1) < 1e-13, a


def kocks_fixed_point(mat):
    # active system: rho_a = 1 / (2 y_c l_a), l_a = K / sqrt(7 rho_a + 4 rho_i)
    # => (2 y_c K rho_a)^2 = 7 rho_a + 4 rho_i, positive root
    rho_i = mat.rho0_total / 12
    c = (2 * mat.yc * mat.K) ** 2
    return (7 + np.sqrt(49 + 16 * c * rho_i)) / (2 * c), rho_i


@pytest.mark.parametrize("yc", [15e-9, 1.5e-6])
def test_kocks_mecking_fixed_point_is_invariant(yc):
    # at rho = 1/(2 y_c l) the implicit update
    #   rho <- (rho + |dgam|/(b l)) / (1 + 2 y_c |dgam| / b)
    # returns rho for every slip increment; a mean free path summed over all
    # systems, or a missing factor 2 on y_c, moves the fixed point
    mat = rvegen.material("Cu", gnd_enabled=False, yc=yc)
    rho_a, rho_i = kocks_fixed_point(mat)
    rve = one_voxel(mat)
    rho = np.full(12, rho_i)
    rho[list(ACTIVE)] = rho_a
    rve.rho_ssd[:] = rho
    for k in range(8):
        info = rve.step(np.array([1e-3, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), 1.0)
        assert info.converged
    assert rve.Fp[0, 0, 0] - 1 > 1e-3                        # it flowed plastically
    assert np.abs(rve.rho_ssd[0] / rho - 1).max() < 1e-13


def test_saturated_flow_stress_of_a_cube_crystal():
    # At the fixed point tauc is constant.  For system 1 (active) the four
    # inactive systems 0, 3, 6, 9 are coplanar, glissile, glissile and Lomer;
    # the eight active ones are self, coplanar, Hirth x2, Lomer, collinear and
    # glissile x2.  The steady flow stress is (tauc / m) (eps_true_rate /
    # (8 m gdot0))^(1/n) with m = 1/sqrt(6).  A larger y_c keeps the
    # saturated stress low (finite-strain terms are O(sigma / E)).
    mat = rvegen.material("Cu", gnd_enabled=False, yc=1.5e-6)
    rho_a, rho_i = kocks_fixed_point(mat)
    rve = one_voxel(mat)
    rve.rho_ssd[:] = rho_i
    rve.rho_ssd[:, list(ACTIVE)] = rho_a
    rate, dt, n_inc = 1e-3, 1.0, 20
    for k in range(n_inc):
        assert rve.step(np.array([rate * dt, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), dt).converged
    qs = {c: Q[c] / Q["self"] for c in Q}
    sum_active = qs["self"] + qs["coplanar"] + 2 * qs["hirth"] + qs["lomer"] + qs["collinear"] + 2 * qs["glissile"]
    sum_inactive = qs["coplanar"] + 2 * qs["glissile"] + qs["lomer"]
    tauc_a = 10.0 + 0.3 * cu_mu() * 0.256e-9 * np.sqrt(sum_active * rho_a + sum_inactive * rho_i)
    tauc, _ = rve.hardening()
    assert np.abs(tauc[0, list(ACTIVE)] / tauc_a - 1).max() < 1e-12
    m = 1.0 / np.sqrt(6.0)
    eps = rate * dt * n_inc
    expected = (tauc_a / m) * (rate / (1 + eps) / (8 * m * mat.gdot0)) ** (1.0 / mat.n)
    _, sig = rve.macro_stress()
    assert abs(sig[0, 0] / expected - 1) < 1.5e-3, (sig[0, 0], expected)


def test_ssd_storage_rate_matches_the_continuous_law():
    # Physical Cu constants, [100] tension in small steps past yield.  The
    # per-system slip of each increment is read from Fp: M = Fp_k Fp_{k-1}^-1
    # has M_11 - 1 = 8 |dgam| / sqrt(6).  The active systems' density must
    # follow d rho / d gamma = (sqrt(7 rho + 4 rho_i) / K - 2 y_c rho) / b
    # (integrated here by scipy) up to the first-order error of the frozen
    # mean free path; a wrong unit or factor on b is off by far more.
    mat = rvegen.material("Cu", gnd_enabled=False)
    rho_i = mat.rho0_total / 12
    rve = one_voxel(mat)
    assert rve.step(np.array([4e-4, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), 0.4).converged
    gam, gs, rho_a = 0.0, [], []
    Fp_old = rve.Fp[0].copy()
    for k in range(60):
        assert rve.step(np.array([2e-5, 0, 0, 0, 0, 0, 0, 0, 0]), MASK, np.zeros(9), 0.02).converged
        M = rve.Fp[0] @ np.linalg.inv(Fp_old)
        Fp_old = rve.Fp[0].copy()
        gam += (M[0, 0] - 1) * np.sqrt(6.0) / 8
        gs.append(gam)
        rho_a.append(rve.rho_ssd[0, list(ACTIVE)].mean())
    assert np.ptp(rve.rho_ssd[0, list(ACTIVE)]) < 1e-9 * rho_a[-1]     # the eight are equivalent
    assert np.abs(rve.rho_ssd[0, list(INACTIVE)] / rho_i - 1).max() < 1e-12
    ode = solve_ivp(lambda g, r: [(np.sqrt(7 * r[0] + 4 * rho_i) / mat.K - 2 * mat.yc * r[0]) / mat.b],
                    (0.0, gs[-1]), [rho_i], t_eval=gs, rtol=1e-11, atol=1.0)
    ratio = np.array(rho_a) / ode.y[0]
    assert rho_a[-1] > 3.5 * rho_i                                      # a real transient
    assert abs(ratio[-1] - 1) < 0.025, ratio[-1]
    assert np.all(np.diff(ratio) < 0) and ratio[-1] > 1               # first-order lag, shrinking


def test_gnd_map_on_a_screw_character_slip_field():
    # Fp = I + gamma(zeta) s (x) m with zeta along t = m x s gives
    # G = -gamma' s (x) s: screw character along s.  The minimum-norm
    # segment densities must equal pinv(A) vec(G), and every system's GND
    # density |rho_edge^a| + 1/2 |rho_screw^d(a)| with d(a) from SCREW_OF.
    mat = rvegen.material("Cu")
    N = 16
    s, m = cr.slip_systems()
    a0 = 0
    wave = np.rint(np.cross(m[a0], s[a0]) * np.sqrt(6.0)).astype(int)   # (-2, 1, 1)
    assert tuple(wave) == (-2, 1, 1)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    gam = 1e-3 * np.sin(2 * np.pi * (wave[0] * x + wave[1] * y + wave[2] * z) / N)
    rve = one_voxel(mat, n=N)
    rve.Fp = np.eye(3)[None] + gam.reshape(-1)[:, None, None] * np.outer(s[a0], m[a0])[None]
    rve.hardening()
    G = rve.G.reshape(-1, 9)
    A = cr.nye_matrix(np.eye(3), mat.b)
    rho18 = G @ np.linalg.pinv(A).T
    assert np.abs(rve.rho18 - rho18).max() < 1e-9 * np.abs(rho18).max()
    screw = np.abs(rho18[:, 12:]).max(axis=0)
    assert screw[SCREW_OF[a0]] == screw.max() and screw.max() > 0.5 * np.abs(rho18).max()
    assert len(set(np.round(screw / screw.max(), 6))) >= 3            # directions distinguishable
    expect = np.abs(rho18[:, :12]) + 0.5 * np.abs(rho18[:, 12 + np.array(SCREW_OF)])
    assert np.abs(rve.rho_gnd - expect).max() < 1e-9 * expect.max()
