"""Pins of the oracle's forward-mode sensitivities d<P_11>/d theta,
theta = (tau0, K, alpha, b), against central finite differences of the
oracle's own stress-strain curve (CPU only).

An 8^3 RVE of 5 Cu grains with a 8 um edge (the GND density matters at this
size), 4 increments of tension: every parameter enters (tau0 and alpha the
Taylor stress, K the mean free path of the SSD storage from the second
increment on, b the GND densities, the Taylor stress and the storage)."""
import dataclasses

import numpy as np
import pytest

import rvegen
from oracle import sensitivity as se
from oracle import solver

MASK = rvegen.UNIAXIAL_X_MASK
WL = rvegen.Workload("s8", 8, 5, "Cu", 0.004, 4, seed=31, L=8e-6)


def curve(mat):
    gid, quat, _ = WL.inputs()
    o = solver.RVE(gid, quat, mat, WL.edge)
    ys = []
    for _ in range(WL.increments):
        assert o.step(WL.dFbar(), MASK, np.zeros(9), WL.dt).converged
        ys.append(o.macro_stress()[0][0, 0])
    return np.array(ys)


@pytest.fixture(scope="module")
def sens():
    gid, quat, mat = WL.inputs()
    s = se.SensitivityRVE(solver.RVE(gid, quat, mat, WL.edge))
    out = []
    for _ in range(WL.increments):
        info, dP = s.step(WL.dFbar(), MASK, np.zeros(9), WL.dt)
        assert info.converged
        out.append(dP)
    return mat, np.array(out)          # (increments, 4, 3, 3)


@pytest.mark.parametrize("j", range(4), ids=se.PARAMS)
@pytest.mark.parametrize("hrel,tol", [(1e-4, 1e-7), (1e-6, 1e-5)], ids=["h1e-4", "h1e-6"])
def test_sensitivity_matches_central_differences(sens, j, hrel, tol):
    mat, dP = sens
    name = se.PARAMS[j]
    v = getattr(mat, name)
    h = hrel * v
    fd = (curve(dataclasses.replace(mat, **{name: v + h})) - curve(dataclasses.replace(mat, **{name: v - h}))) / (2 * h)
    g = dP[:, j, 0, 0]
    assert np.abs(fd - g).max() <= tol * np.abs(g).max()


def test_sensitivity_structure(sens):
    """K (the mean-free-path constant) acts only through the SSD storage of
    earlier increments, so the first increment does not depend on it; the
    stress-controlled means stay at their prescribed zero."""
    _, dP = sens
    assert dP[0, 1, 0, 0] == 0.0
    assert np.abs(dP[1:, 1, 0, 0]).min() > 0
    stress_ctl = (MASK == 0).reshape(3, 3)
    assert np.abs(dP[:, :, stress_ctl]).max() < 1e-9 * np.abs(dP[:, :, 0, 0]).max()
