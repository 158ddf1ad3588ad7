"""Sensitivities of the stress-strain curve with respect to (tau0, K, alpha, b)
through the C ABI: against the oracle's forward-mode sensitivities, against
central differences of the GPU path itself, through the autograd Function
(a loss whose target curve is the forward run at theta* has zero gradient
there), in mixed precision, and only after a converged increment."""
import dataclasses

import numpy as np
import pytest

import rvegen
from oracle import sensitivity as se
from oracle import solver

pytestmark = pytest.mark.gpu
MASK = rvegen.UNIAXIAL_X_MASK
WL = rvegen.Workload("s8", 8, 5, "Cu", 0.004, 4, seed=31, L=8e-6)


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


def gpu_run(pkg, mat, sens=True, **opts):
    gid, quat, _ = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, **opts)
    if sens:
        r.enable_sensitivity()
    ys, ds = [], []
    for _ in range(WL.increments):
        assert r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)["converged"]
        ys.append(r.macro_stress()[0][0, 0])
        if sens:
            ds.append(r.stress_sensitivity())
    r.close()
    return np.array(ys), (np.array(ds) if sens else None)


@pytest.fixture(scope="module")
def oracle_sens():
    gid, quat, mat = WL.inputs()
    s = se.SensitivityRVE(solver.RVE(gid, quat, mat, WL.edge))
    out = []
    for _ in range(WL.increments):
        info, dP = s.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)
        assert info.converged
        out.append(dP)
    return mat, np.array(out)


def test_sensitivity_matches_oracle(pkg, oracle_sens):
    mat, ref = oracle_sens
    _, g = gpu_run(pkg, mat)
    for j in range(4):
        scale = np.abs(ref[:, j]).max()
        assert np.abs(g[:, j] - ref[:, j]).max() <= 1e-7 * scale, pkg.PARAMS[j]


@pytest.mark.parametrize("j", range(4), ids=["tau0", "K", "alpha", "b"])
def test_sensitivity_matches_gpu_central_differences(pkg, oracle_sens, j):
    mat, _ = oracle_sens
    _, g = gpu_run(pkg, mat)
    name = pkg.PARAMS[j]
    v = getattr(mat, name)
    for hrel, tol in ((1e-4, 1e-7), (1e-6, 1e-5)):
        h = hrel * v
        yp, _ = gpu_run(pkg, dataclasses.replace(mat, **{name: v + h}), sens=False)
        ym, _ = gpu_run(pkg, dataclasses.replace(mat, **{name: v - h}), sens=False)
        fd = (yp - ym) / (2 * h)
        assert np.abs(fd - g[:, j, 0, 0]).max() <= tol * np.abs(g[:, j, 0, 0]).max(), (name, hrel)


def test_autograd_gradient_of_calibration_loss(pkg, oracle_sens):
    """J(theta) = sum_k (<P_11>_k(theta) - y*_k)^2 with y* the curve at
    theta* = theta (1 + 0.05 u), u seeded in [-1, 1]: grad J(theta*) = 0, and at
    theta the gradient equals the oracle's 2 (y - y*)^T dy/dtheta."""
    import torch
    from paper_1910_01946_gb300.autograd import stress_strain_curve
    mat, ref = oracle_sens
    gid, quat, _ = WL.inputs()
    theta0 = np.array([getattr(mat, n) for n in pkg.PARAMS])
    u = np.random.default_rng(7).uniform(-1, 1, 4)
    theta_star = theta0 * (1 + 0.05 * u)
    args = (gid, quat, mat, WL.edge, WL.dFbar(), MASK, WL.dt, WL.increments)
    with torch.no_grad():
        target = stress_strain_curve(torch.tensor(theta_star), *args)
    ts = torch.tensor(theta_star, requires_grad=True)
    loss = ((stress_strain_curve(ts, *args) - target) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == 0.0 and np.all(ts.grad.numpy() == 0.0)
    t0 = torch.tensor(theta0, requires_grad=True)
    y = stress_strain_curve(t0, *args)
    loss = ((y - target) ** 2).sum()
    loss.backward()
    g_oracle = 2.0 * (y.detach().numpy() - target.numpy()) @ ref[:, :, 0, 0]
    assert np.allclose(t0.grad.numpy(), g_oracle, rtol=1e-6, atol=0)


def test_mixed_precision_sensitivity_matches_fp64(pkg, oracle_sens):
    mat, ref = oracle_sens
    _, g = gpu_run(pkg, mat, precision=1)
    for j in range(4):
        assert np.abs(g[:, j] - ref[:, j]).max() <= 1e-6 * np.abs(ref[:, j]).max(), pkg.PARAMS[j]


def test_sensitivity_needs_a_converged_increment(pkg, oracle_sens):
    """No sensitivity before a converged increment; a failed step (max_newton
    = 1) commits nothing and reports none."""
    mat, _ = oracle_sens
    gid, quat, _ = WL.inputs()
    r = pkg.RVE(gid, quat, mat, WL.edge, max_newton=1)
    r.enable_sensitivity()
    with pytest.raises(pkg.RVEError):
        r.stress_sensitivity()
    info = r.step(WL.dFbar(), MASK, np.zeros(9), WL.dt, check=False)
    assert info["status"] != 0
    with pytest.raises(pkg.RVEError):
        r.stress_sensitivity()
    r.close()
