"""The macroscopic stress-strain curve as a differentiable function of the
material parameters theta = (tau0, K, alpha, b), for calibrating them against
measured curves (the paper fits its parameters to Hall-Petch data, Sec. 4).

The forward pass runs the load history on the GPU with the library's
forward-mode sensitivities switched on (rve_sensitivity_enable): every
increment also returns d<P_11>/d theta, so the Jacobian of the whole curve is
known when the forward pass ends, and backward is one small product with it.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import PARAMS, RVE


class StressStrainCurve(torch.autograd.Function):
    """theta (4,) float64 -> <P_11> after each increment (increments,)."""

    @staticmethod
    def forward(ctx, theta, grain_id, quat, mat, L, dFbar, mask, dt, increments, options):
        th = theta.detach().cpu().to(torch.float64).numpy()
        m = dataclasses.replace(mat, **{name: float(th[j]) for j, name in enumerate(PARAMS)})
        r = RVE(grain_id, quat, m, L, **(options or {}))
        ys, jac = [], []
        try:
            r.enable_sensitivity()
            for _ in range(increments):
                r.step(dFbar, mask, np.zeros(9), dt)
                ys.append(r.macro_stress()[0][0, 0])
                jac.append(r.stress_sensitivity()[:, 0, 0])
        finally:
            r.close()
        J = torch.tensor(np.array(jac), dtype=torch.float64)
        ctx.save_for_backward(J)
        return torch.tensor(ys, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_curve):
        (J,) = ctx.saved_tensors
        return (J.t() @ grad_curve.to(J.dtype),) + (None,) * 9


def stress_strain_curve(theta, grain_id, quat, mat, L, dFbar, mask, dt, increments, **options):
    """Differentiable <P_11> curve of an RVE under the given loading; `mat` is
    a material record whose tau0, K, alpha and b are replaced by theta."""
    return StressStrainCurve.apply(theta, grain_id, quat, mat, L, dFbar, mask, dt, increments, options)
