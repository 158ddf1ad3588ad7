"""Failure paths of rve_step, each made on the host (no GPU fault is ever
provoked): a load the local update cannot follow, a non-finite state, a
linear solve that cannot reach its tolerance, and the bounded wait of the
staged FP32 tangent apply run out on purpose.  Every failed step must return
its status, leave the last committed increment untouched, and leave a handle
that completes a normal step afterwards."""
import numpy as np
import pytest

import rvegen

pytestmark = pytest.mark.gpu

MASK = rvegen.UNIAXIAL_X_MASK
WL = rvegen.Workload("cu8", 8, 5, "Cu", 0.004, 4, seed=31)


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


def committed(r):
    return {k: r.field(k) for k in ("F", "P", "FP", "S", "RHO_SSD")}


def assert_same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def fresh_first_step(pkg, **opts):
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, **opts)
    assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
    out = committed(r)
    r.close()
    return out


def test_local_nonconvergence_on_an_oversized_load(pkg):
    # 50 % strain in one increment needs slip increments above the local cap
    # (|dgam| <= 0.1): no voxel update exists, the step is refused
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge)
    before = committed(r)
    big = np.zeros(9); big[0] = 0.5
    info = r.step(big, MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] == pkg.RVE_ENOCONV_LOCAL and not info["converged"]
    assert info["local_failures"] > 0
    assert_same(committed(r), before)
    assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
    assert_same(committed(r), fresh_first_step(pkg))
    r.close()


def test_local_nonconvergence_with_one_local_iteration(pkg):
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, max_local=1)
    before = committed(r)
    info = r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] == pkg.RVE_ENOCONV_LOCAL and info["local_failures"] > 0
    assert_same(committed(r), before)
    r.close()


def test_non_finite_state_is_reported(pkg):
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge)
    before = committed(r)
    F = before["F"].copy()
    F[3, 2, 5, 0] = np.nan
    r.set_field("F", F)
    info = r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] == pkg.RVE_ENAN and not info["converged"]
    after = committed(r)
    for k in ("FP", "S", "RHO_SSD", "P"):
        assert np.array_equal(after[k], before[k]), k
    assert np.isnan(after["F"][3, 2, 5, 0])          # the state is what was set, nothing committed
    r.set_field("F", before["F"])
    assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
    assert_same(committed(r), fresh_first_step(pkg))
    r.close()


def test_unreachable_linear_solve_is_reported(pkg):
    # the sensitivity solves (CG, then BiCGStab) at an unreachable tolerance
    # both stop at max_cg: the step fails with RVE_ENOCONV_CG before its commit
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, max_cg=400)
    before = committed(r)
    r.enable_sensitivity(tol=1e-300)
    info = r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] == pkg.RVE_ENOCONV_CG and not info["converged"]
    assert_same(committed(r), before)
    r.enable_sensitivity()                              # default tolerance
    assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
    assert np.isfinite(r.stress_sensitivity()).all()
    r.close()


def test_staged_apply_wait_limit_runs_out_and_recovers(pkg):
    # mixed precision with the bulk-copy tangent apply: a per-tile wait limit
    # of 0 polls makes every block give up at its first wait; each block still
    # waits (at the default limit) for the copies it issued before it leaves
    gid, quat, mat = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, precision=1, tma=1)
    assert r.tuning()["tma"]
    before = committed(r)
    r.set_wait_limit(0)
    info = r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] == pkg.RVE_ETIMEOUT and not info["converged"]
    assert_same(committed(r), before)
    r.set_wait_limit(1 << 22)
    assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
    assert_same(committed(r), fresh_first_step(pkg, precision=1, tma=1))
    r.close()
