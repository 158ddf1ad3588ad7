"""GPU path (librve.so through its C ABI) against the FP64 oracle on the same
seeded inputs: each step of the increment on its own (projection, Nye curl and
hardening, local update and tangent), whole increments on small RVEs, and
sampled outputs on the 64^3 / 100-grain workload the benchmark times.

Tolerance.  Single kernels are compared as max|gpu - oracle| / max|oracle|
per field and agree to round-off (1e-11 .. 1e-13).  Whole increments are
compared per component on the informative part of each field (F - I, Fp - I,
rho_SSD - rho_0, P, sigma, rho_GND): max|gpu - oracle| over the component's
own max|oracle|, floored at 1e-3 of the field's largest component, against
the 1e-9 relative bound (both sides converge the same discrete equations to
a relative residual of 1e-11, so their difference is the conditioning times
that residual plus round-off)."""
import numpy as np
import pytest

import rvegen
from oracle import constitutive as co
from oracle import crystal as cr
from oracle import solver
from oracle import spectral as sp

pytestmark = pytest.mark.gpu

MASK = rvegen.UNIAXIAL_X_MASK


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1910_01946_gb300 import _build
    _build.build()
    import paper_1910_01946_gb300 as p
    p.load_library()
    return p


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


EYE9 = np.eye(3).reshape(9)


def comp_err(g, o, base=None):
    """Largest per-component relative error of field g against o (last axis =
    components) after subtracting `base` from both (the part that carries
    the information: F - I, Fp - I, rho - rho_0)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    nc = o.shape[-1]
    g = g.reshape(-1, nc)
    o = o.reshape(-1, nc)
    if base is not None:
        g = g - base
        o = o - base
    scale = np.abs(o).max(axis=0)
    den = np.maximum(scale, 1e-3 * scale.max())
    return float((np.abs(g - o).max(axis=0) / den).max())


def check_increment_fields(g, o, tol=1e-9):
    shape = g.shape
    rho0 = o.mat.rho0_total / 12
    assert comp_err(g.field("F"), to_field(o.F, shape), EYE9) < tol, "F - I"
    assert comp_err(g.field("FP"), to_field(o.Fp, shape), EYE9) < tol, "Fp - I"
    assert comp_err(g.field("P"), to_field(o.P, shape)) < tol, "P"
    sig = o.P @ np.swapaxes(o.F, 1, 2) / np.linalg.det(o.F)[:, None, None]
    assert comp_err(g.field("SIGMA"), to_field(sig, shape)) < tol, "sigma"
    assert comp_err(g.field("RHO_SSD"), o.rho_ssd.reshape(shape + (12,)), rho0) < tol, "rho_SSD - rho_0"
    assert comp_err(g.field("RHO_GND"), o.rho_gnd.reshape(shape + (12,))) < tol, "rho_GND"
    Pg, sg = g.macro_stress()
    Po, so = o.macro_stress()
    assert relerr(Pg, Po) < tol and relerr(sg, so) < tol


def to_field(a, shape):
    """(nv, 3, 3) oracle -> (n2, n1, n0, 9)."""
    return a.reshape(shape + (9,))


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 12, 16), (9, 4, 6), (1, 4, 4), (16, 16, 16),
                                   (2, 6, 32), (3, 4, 64), (2, 6, 96), (1, 2, 128)])
def test_projection_matches_oracle(pkg, shape):
    """n0 = 32, 64, 96, 128 take the row-strip stencils (one warp per x line,
    1-4 points per lane); the other widths the tiled ones."""
    import torch
    n2, n1, n0 = shape
    gid = np.zeros(shape, dtype=np.int32)
    r = pkg.RVE(gid, np.array([[1.0, 0, 0, 0]]), rvegen.material("Cu"), 1e-5)
    rng = np.random.default_rng(sum(shape))
    X = rng.standard_normal(shape + (3, 3))
    for mask in (MASK, np.zeros(9, np.uint8), np.ones(9, np.uint8)):
        ref = sp.project(X, mask, r.opt.L / n0)
        Xd = torch.from_numpy(np.ascontiguousarray(np.moveaxis(X.reshape(shape + (9,)), -1, 0).reshape(9, -1))).cuda()
        Y = r.project(mask, Xd).cpu().numpy().reshape((9,) + shape)
        assert relerr(np.moveaxis(Y, 0, -1), ref.reshape(shape + (9,))) < 1e-13
    r.close()


def test_nye_gnd_hardening_match_oracle(pkg):
    wl = rvegen.Workload("t", 12, 5, "Cu", 0.001, 1, seed=9)
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge)
    o = solver.RVE(gid, quat, mat, wl.edge)
    rng = np.random.default_rng(3)
    Fp = np.eye(3) + 2e-3 * rng.standard_normal(gid.shape + (3, 3))
    rho = (1e12 / 12) * (1 + rng.random(gid.shape + (12,)))
    g.set_field("FP", Fp.reshape(gid.shape + (9,)))
    g.set_field("RHO_SSD", rho)
    o.Fp = Fp.reshape(-1, 3, 3).copy()
    o.rho_ssd = rho.reshape(-1, 12).copy()
    g.eval_hardening()
    tauc, ell = o.hardening()
    assert relerr(g.field("NYE"), to_field(o.G, gid.shape)) < 1e-11
    assert relerr(g.field("RHO_GND18"), o.rho18.reshape(gid.shape + (18,))) < 1e-11
    assert relerr(g.field("RHO_GND"), o.rho_gnd.reshape(gid.shape + (12,))) < 1e-11
    assert relerr(g.field("TAUC"), tauc.reshape(gid.shape + (12,))) < 1e-13
    g.close()


def test_constitutive_and_tangent_match_oracle(pkg):
    wl = rvegen.Workload("t", 8, 6, "Cu", 0.001, 1, seed=19)
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge)
    o = solver.RVE(gid, quat, mat, wl.edge)
    rng = np.random.default_rng(5)
    F = np.eye(3) + np.diag([2e-3, -6e-4, -6e-4]) + 1e-3 * rng.standard_normal(gid.shape + (3, 3))
    Fp = np.eye(3) + 1e-3 * rng.standard_normal(gid.shape + (3, 3))
    g.set_field("F", F.reshape(gid.shape + (9,)))
    g.set_field("FP", Fp.reshape(gid.shape + (9,)))
    o.Fp = Fp.reshape(-1, 3, 3).copy()
    dt = 1.0
    it, nf = g.eval_constitutive(dt)
    assert nf == 0
    tauc, _ = o.hardening()
    P, K, S, M, dg, lit, lf = o.constitutive(F.reshape(-1, 3, 3), tauc, np.zeros_like(o.S), dt)
    assert lf == 0 and np.abs(dg).max() > 1e-3          # well into the plastic range
    assert relerr(g.field("P_EVAL"), to_field(P, gid.shape)) < 1e-11
    assert relerr(g.field("DGAM"), dg.reshape(gid.shape + (12,))) < 1e-9
    S6 = np.stack([S[:, i, j] for i, j in co.VP], axis=-1)
    assert relerr(g.field("S_EVAL"), S6.reshape(gid.shape + (6,))) < 1e-11
    assert relerr(g.field("TANGENT"), K.reshape(gid.shape + (81,))) < 1e-10
    g.close()


def run_both(pkg, wl, n_inc, gpu_opts=None):
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge, **(gpu_opts or {}))
    o = solver.RVE(gid, quat, mat, wl.edge)
    curve = []
    for k in range(n_inc):
        gi = g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        oi = o.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert gi["converged"] and oi.converged
        curve.append((g.macro_stress()[0][0, 0], o.macro_stress()[0][0, 0]))
    return g, o, curve


@pytest.mark.parametrize("wl", [rvegen.Workload("cu8", 8, 5, "Cu", 0.004, 4, seed=31),
                                rvegen.Workload("al12", 12, 7, "Al", 0.003, 3, seed=32)],
                         ids=["cu8x4", "al12x3"])
def test_increments_match_oracle(pkg, wl):
    g, o, curve = run_both(pkg, wl, wl.increments)
    check_increment_fields(g, o)
    for a, b in curve:
        assert abs(a - b) < 1e-9 * abs(b)
    assert o.rho_gnd.max() > 0 and np.abs(o.Fp - np.eye(3)).max() > 1e-4
    g.close()


def test_cu16_first_increments_match_oracle(pkg):
    wl = rvegen.WORKLOADS["cu16"]
    g, o, curve = run_both(pkg, wl, 3)
    check_increment_fields(g, o)
    g.close()


@pytest.mark.parametrize("shape", [(24, 24, 6), (6, 24, 24), (32, 8, 6), (64, 6, 4)],
                         ids=["24x24x6", "6x24x24", "32x8x6", "64x6x4"])
def test_increments_match_oracle_mixed_radix_grid(pkg, shape):
    """Grids whose FFT plans chain radix-4, radix-2 and radix-3 passes
    (24 = 4 * 2 * 3), on the x and y axes or on the y and z axes: the plan
    family of the 48^3 and 96^3 sweep RVEs; and x lines of 32 and 64 voxels,
    which take the row-strip stencils.  Three increments to 6e-4 (past the
    plastic onset, GND active)."""
    n0, n1, n2 = shape
    ng = 6
    gid, _ = rvegen.voronoi_grain_map(0, ng, 2401, shape=shape)
    quat = rvegen.random_quaternions(ng, 2401 + 7919)
    mat = rvegen.material("Cu")
    L = 20e-6 * (np.pi * ng / 6.0) ** (1.0 / 3.0)
    g = pkg.RVE(gid, quat, mat, L)
    o = solver.RVE(gid, quat, mat, L)
    d = np.zeros(9); d[0] = 2e-4
    for k in range(3):
        assert g.step(d, MASK, np.zeros(9), 0.2)["converged"]
        assert o.step(d, MASK, np.zeros(9), 0.2).converged
    check_increment_fields(g, o)
    assert o.rho_gnd.max() > 0 and np.abs(o.Fp - np.eye(3)).max() > 5e-4
    g.close()


def test_failed_step_leaves_state_and_handle_usable(pkg):
    wl = rvegen.Workload("t", 8, 4, "Cu", 0.002, 2, seed=41)
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge, max_newton=1)
    F0 = g.field("F")
    info = g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt, check=False)
    assert info["status"] == pkg.RVE_ENOCONV_NEWTON and not info["converged"]
    assert np.array_equal(g.field("F"), F0)
    g.close()
    g = pkg.RVE(gid, quat, mat, wl.edge)
    info = g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    assert info["converged"]
    # NaN load is rejected before touching the device
    bad = wl.dFbar(); bad[0] = np.nan
    assert g.step(bad, MASK, np.zeros(9), wl.dt, check=False)["status"] == pkg.RVE_EINVAL
    # checkpoint / restore round trip
    buf = g.checkpoint()
    F1 = g.field("F")
    g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    g.restore(buf)
    assert np.array_equal(g.field("F"), F1)
    corrupt = buf.copy(); corrupt[0] ^= 0xFF
    with pytest.raises(pkg.RVEError):
        g.restore(corrupt)
    g.close()


@pytest.mark.parametrize("n_inc", [2, 12])
def test_full_size_workload_sampled(pkg, n_inc):
    """64^3, 100 grains, Cu (the benchmark workload, in the launch
    configuration the benchmark times), 2 or 12 increments (0.2 % and 1.2 %
    strain, the second well into plastic flow) on the GPU; the oracle
    recomputes the hardening on the full field and the local update and
    tangent at sampled voxels from the GPU's state, and checks the
    equilibrium and macro invariants on the full field."""
    wl = rvegen.WORKLOADS["cu64"]
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge)
    for k in range(n_inc):
        info = g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert info["converged"]
    o = solver.RVE(gid, quat, mat, wl.edge)
    nv = gid.size
    F = g.field("F").reshape(nv, 3, 3)
    P = g.field("P").reshape(nv, 3, 3)
    # macro invariants
    Fm = F.mean(axis=0).reshape(9)
    assert np.allclose(Fm[MASK == 1], (np.eye(3).reshape(9) + n_inc * wl.dFbar())[MASK == 1], atol=1e-14)
    Pm = P.mean(axis=0).reshape(9)
    assert np.abs(Pm[MASK == 0]).max() < 1e-9 * np.abs(Pm).max()
    R = sp.project(P.reshape(gid.shape + (3, 3)), MASK, o.h)
    assert np.sqrt(np.mean(R ** 2)) < 1e-10 * np.abs(Pm).max()
    # the GPU's committed P at sampled voxels equals the oracle's local update
    # from the GPU's state at the start of the increment is not recoverable
    # after commit, so sample the hardening and one fresh local evaluation
    Fp = g.field("FP").reshape(nv, 3, 3)
    rho = g.field("RHO_SSD").reshape(nv, 12)
    o.Fp, o.rho_ssd = Fp.copy(), rho.copy()
    g.eval_hardening()
    tauc, _ = o.hardening()
    assert relerr(g.field("TAUC").reshape(nv, 12), tauc) < 1e-12
    assert relerr(g.field("RHO_GND").reshape(nv, 12), o.rho_gnd) < 1e-10
    dt = wl.dt
    g.eval_constitutive(dt)
    rng = np.random.default_rng(0)
    sample = rng.choice(nv, 512, replace=False)
    Pe = g.field("P_EVAL").reshape(nv, 3, 3)
    Ke = g.field("TANGENT").reshape(nv, 3, 3, 3, 3)
    for gr in o.grains:
        sel = np.intersect1d(gr["idx"], sample)
        if len(sel) == 0:
            continue
        r = co.local_update(F[sel], Fp[sel], tauc[sel], np.zeros((len(sel), 3, 3)), gr["C"], gr["S0"], dt,
                            mat.gdot0, mat.n, 1e-14 * o.mu)
        assert relerr(Pe[sel], r.P) < 1e-10
        assert relerr(Ke[sel], r.K) < 1e-9
    g.close()


@pytest.mark.parametrize("wl", [rvegen.Workload("cu8", 8, 5, "Cu", 0.004, 4, seed=31)], ids=["cu8x4"])
def test_mixed_precision_increments_match_oracle(pkg, wl):
    """precision = 1: FP32 conjugate gradients, FP64 local update and residual.
    Newton converges the FP64 residual, so the increment is the FP64 one."""
    g, o, curve = run_both(pkg, wl, wl.increments, gpu_opts=dict(precision=1))
    check_increment_fields(g, o)
    assert g.field("TANGENT").dtype == np.float64
    g.close()


def test_mixed_precision_matches_fp64_path_cu16(pkg):
    wl = rvegen.WORKLOADS["cu16"]
    gid, quat, mat = wl.inputs()
    a = pkg.RVE(gid, quat, mat, wl.edge)
    b = pkg.RVE(gid, quat, mat, wl.edge, precision=1)
    for k in range(4):
        ia = a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        ib = b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    for name, base in (("F", EYE9), ("P", None), ("FP", EYE9), ("RHO_GND", None), ("SIGMA", None)):
        assert comp_err(b.field(name), a.field(name), base) < 1e-9, name
    assert relerr(b.macro_stress()[0], a.macro_stress()[0]) < 1e-9
    a.close(); b.close()


@pytest.mark.parametrize("wl", [rvegen.Workload("cu8", 8, 5, "Cu", 0.004, 4, seed=31)], ids=["cu8x4"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_bicgstab_increments_match_oracle(pkg, wl, precision):
    """krylov = 1 solves every Newton step with BiCGStab instead of CG; the
    converged increment is the same one the oracle's CG path reaches."""
    gid, quat, mat = wl.inputs()
    g = pkg.RVE(gid, quat, mat, wl.edge, krylov=1, precision=precision)
    o = solver.RVE(gid, quat, mat, wl.edge)
    for k in range(wl.increments):
        gi = g.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        oi = o.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert gi["converged"] and oi.converged
        assert gi["bicgstab_solves"] == gi["newton_iters"]
    check_increment_fields(g, o)
    g.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_row_strip_stencils_match_tiled(pkg, precision):
    """The row-strip stencils (default where n0 = 32 k) and the tiled ones
    (stencils = 1) reach the same increments on the 64^3 workload."""
    wl = rvegen.WORKLOADS["cu64"]
    gid, quat, mat = wl.inputs()
    a = pkg.RVE(gid, quat, mat, wl.edge, precision=precision, stencils=0)
    b = pkg.RVE(gid, quat, mat, wl.edge, precision=precision, stencils=1)
    for k in range(3):
        assert a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
        assert b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
    for name, base in (("F", EYE9), ("P", None), ("FP", EYE9), ("RHO_GND", None)):
        assert comp_err(a.field(name), b.field(name), base) < 1e-9, name
    a.close(); b.close()


def test_staged_tangent_apply_matches_plain_loads(pkg):
    """Mixed precision: the tangent apply staged through shared memory by bulk
    asynchronous copies (tma = 1, one persistent block per SM) and the plain
    per-thread loads (tma = 0) reach the same FP64 increment."""
    wl = rvegen.WORKLOADS["cu16"]
    gid, quat, mat = wl.inputs()
    a = pkg.RVE(gid, quat, mat, wl.edge, precision=1, tma=1)
    b = pkg.RVE(gid, quat, mat, wl.edge, precision=1, tma=0)
    for k in range(3):
        assert a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
        assert b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
    for name, base in (("F", EYE9), ("P", None), ("FP", EYE9), ("RHO_GND", None)):
        assert comp_err(a.field(name), b.field(name), base) < 1e-9, name
    a.close(); b.close()


def test_nye_schemes_match_oracle_and_show_gibbs_ringing(pkg):
    """rve_eval_nye on a bicrystal whose Fp jumps across the slab boundaries
    (App. B): the rotated scheme against the oracle's stencil (exactly local
    to the boundary layers), the standard spectral derivative against the
    oracle's FFT form (Gibbs oscillations through the grains)."""
    n = 32
    Fp = rvegen.bicrystal_slip_jump(n)
    gid = np.zeros((n, n, n), dtype=np.int32)
    g = pkg.RVE(gid, np.array([[1.0, 0, 0, 0]]), rvegen.material("Cu"), 20e-6)
    g.set_field("FP", Fp.reshape(gid.shape + (9,)))
    h = 20e-6 / n
    g.eval_nye(0)
    Gr = g.field("NYE")
    g.eval_nye(1)
    Gs = g.field("NYE")
    ref_r = sp.nye_tensor(Fp, h).reshape(gid.shape + (9,))
    ref_s = sp.nye_tensor_standard(Fp, h).reshape(gid.shape + (9,))
    assert relerr(Gr, ref_r) < 1e-12
    assert relerr(Gs, ref_s) < 1e-12
    col_r = np.abs(Gr).max(axis=(0, 1, 3))
    col_s = np.abs(Gs).max(axis=(0, 1, 3))
    assert np.abs(col_r[[x for x in range(n) if x not in (n // 2 - 1, n - 1)]]).max() < 1e-12 * col_r.max()
    assert col_s[[n // 4, 3 * n // 4]].min() > 0.1 * col_s.max()
    with pytest.raises(pkg.RVEError):
        g.eval_nye(2)
    g.close()


def test_load_continuation_reaches_the_same_increment(pkg):
    """A direct Newton solve held to 6 iterations fails at the plastic onset
    (it needs 16); the load continuation solves the same increment in stages
    (8, each within 6 iterations).  The
    converged increment equals the one a direct solve reaches (and the
    oracle's)."""
    wl = rvegen.Workload("cu8", 8, 5, "Cu", 0.004, 4, seed=31)
    gid, quat, mat = wl.inputs()
    a = pkg.RVE(gid, quat, mat, wl.edge, max_newton=6, continuation=6)
    b = pkg.RVE(gid, quat, mat, wl.edge, continuation=0)
    o = solver.RVE(gid, quat, mat, wl.edge)
    staged = 0
    for k in range(2):
        ia = a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        ib = b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert o.step(wl.dFbar(), MASK, np.zeros(9), wl.dt).converged
        assert ia["converged"] and ib["converged"] and ib["load_stages"] == 1
        staged = max(staged, ia["load_stages"])
    assert staged > 1
    for name, base in (("F", EYE9), ("P", None), ("FP", EYE9), ("RHO_SSD", None)):
        assert comp_err(a.field(name), b.field(name), base) < 1e-9, name
    check_increment_fields(a, o)
    a.close(); b.close()
