"""Spectral operators of the oracle (test infrastructure only).

Axis convention: a field array has numpy shape (n2, n1, n0, ...) so that x
(axis 2) is the fastest voxel index; voxels are cubes of edge h.

* Rotated-scheme derivative (App. A, Eqs. derivative2 and kas).  The
  modified frequency k_i(xi) = 1/4 tan(xi_i/2) prod_j (1 + e^{i xi_j}) turns the
  derivative into the symbol i k_i / h.  Since tan(x/2) (1 + e^{ix}) = -i (e^{ix} - 1),
  this symbol equals (1/4h)(e^{i xi_i} - 1) prod_{j != i}(1 + e^{i xi_j}); with the
  DFT convention f^(xi) = sum_n f(n) e^{-i xi n} a factor e^{i xi_j} is a shift by one
  voxel along j, so the operator is exactly the real-space stencil "difference
  along e_i averaged over the four voxel edges parallel to e_i" whose result sits
  at the voxel corner n + (1/2, 1/2, 1/2) and is stored at index n.  The oracle
  applies that stencil directly (no FFT) for the Nye tensor.
  Frequencies: the paper writes xi for odd N only (Eq. freqs); the reading used
  is xi = 2 pi fftfreq(N) for any N.
* Nye tensor (Eq. Nye_finite_strain, App. B): the reading used is
  G_ij = - eps_jkl d_k Fp_il  (i: Burgers index = row of Fp, j: line index),
  consistent with G_ij = sum_a rho^a b_i^a t_j^a (Eq. defA).
* Standard spectral derivative (i xi / h, App. A's continuous frequencies),
  for the Nye tensor only, to show the Gibbs oscillations of App. B.
* Galerkin projection with mixed control (Sec. 2.2, Eqs. weakarbi,
  eql_discrete2): for xi != 0 the compatible projection
  (G X)^_ij = D_j sum_l X^_il conj(D_l) / sum_m |D_m|^2 with D the derivative
  symbol above (a mode whose symbol vanishes, i.e. two or more Nyquist
  components, is zeroed); at xi = 0 the stress-controlled components are kept
  and the strain-controlled ones zeroed.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

LEVI = np.zeros((3, 3, 3))
LEVI[0, 1, 2] = LEVI[1, 2, 0] = LEVI[2, 0, 1] = 1.0
LEVI[0, 2, 1] = LEVI[2, 1, 0] = LEVI[1, 0, 2] = -1.0

_WORKERS = os.cpu_count() or 1


def _shift(f, d0, d1, d2):
    """f(n + (d0, d1, d2)) with periodic wrap; d0 along x (axis 2)."""
    return np.roll(f, (-d2, -d1, -d0), axis=(0, 1, 2))


def stencil_derivative(f, axis, h):
    """Rotated-scheme derivative along x (axis=0), y (1) or z (2); see module doc."""
    others = [a for a in range(3) if a != axis]
    out = np.zeros_like(f)
    for o1 in (0, 1):
        for o2 in (0, 1):
            lo = [0, 0, 0]
            lo[others[0]] = o1
            lo[others[1]] = o2
            hi = list(lo)
            hi[axis] += 1
            out += _shift(f, *hi) - _shift(f, *lo)
    return out / (4.0 * h)


def nye_tensor(Fp, h):
    """G_ij = - eps_jkl d_k Fp_il for Fp of shape (n2, n1, n0, 3, 3)."""
    dFp = np.stack([stencil_derivative(Fp, k, h) for k in range(3)], axis=-1)  # [..., i, l, k]
    return -np.einsum("jkl,...ilk->...ij", LEVI, dFp)


def standard_frequencies(n):
    """xi = 2 pi fftfreq(n), with the Nyquist entry of an even n set to 0 (its
    derivative has no real representation): the continuous frequencies that
    App. A contrasts with the rotated scheme."""
    xi = 2.0 * np.pi * np.fft.fftfreq(n)
    if n % 2 == 0:
        xi[n // 2] = 0.0
    return xi


def nye_tensor_standard(Fp, h):
    """G_ij = - eps_jkl d_k Fp_il with the standard spectral derivative
    d_k <-> i xi_k / h (the trigonometric interpolant's derivative), for the
    comparison of App. B: at a jump of Fp across a grain boundary it rings
    (Gibbs oscillations), where the rotated stencil of nye_tensor stays local."""
    n2, n1, n0 = Fp.shape[:3]
    Fh = np.fft.fftn(Fp, axes=(0, 1, 2))
    xs = (standard_frequencies(n0)[None, None, :], standard_frequencies(n1)[None, :, None],
          standard_frequencies(n2)[:, None, None])
    dFp = np.stack([np.real(np.fft.ifftn(1j * xs[k][..., None, None] / h * Fh, axes=(0, 1, 2)))
                    for k in range(3)], axis=-1)                              # [..., i, l, k]
    return -np.einsum("jkl,...ilk->...ij", LEVI, dFp)


def _unit_phase(n):
    """e^{i xi} for xi = 2 pi fftfreq(n), exactly -1 at the Nyquist index."""
    w = np.exp(2j * np.pi * np.fft.fftfreq(n))
    if n % 2 == 0:
        w[n // 2] = -1.0
    return w


def derivative_symbols(shape, h, half=True):
    """(D0, D1, D2): symbols of the rotated-scheme derivative along x, y, z on the
    (half, when half=True) spectrum grid of a field of numpy shape (n2, n1, n0)."""
    n2, n1, n0 = shape
    w0 = _unit_phase(n0)
    if half:
        w0 = w0[: n0 // 2 + 1]
    w1, w2 = _unit_phase(n1), _unit_phase(n2)
    W0, W1, W2 = w0[None, None, :], w1[None, :, None], w2[:, None, None]
    D0 = (W0 - 1) * (1 + W1) * (1 + W2) / (4 * h)
    D1 = (1 + W0) * (W1 - 1) * (1 + W2) / (4 * h)
    D2 = (1 + W0) * (1 + W1) * (W2 - 1) / (4 * h)
    return D0, D1, D2


def project(X, strain_mask, h=1.0):
    """Galerkin projection with mixed control of a tensor field X (n2, n1, n0, 3, 3)."""
    shape = X.shape[:3]
    Xh = sfft.rfftn(X, axes=(0, 1, 2), workers=_WORKERS)
    D = np.stack(derivative_symbols(shape, h), axis=-1)          # (..., 3) complex
    d2 = np.sum(np.abs(D) ** 2, axis=-1)
    s = np.einsum("...il,...l->...i", Xh, np.conj(D))
    with np.errstate(invalid="ignore", divide="ignore"):
        Gh = np.einsum("...j,...i->...ij", D, s) / d2[..., None, None]
    Gh[d2 == 0.0] = 0.0
    keep = (np.asarray(strain_mask).reshape(3, 3) == 0)
    Gh[0, 0, 0] = np.where(keep, Xh[0, 0, 0], 0.0)
    return sfft.irfftn(Gh, s=shape, axes=(0, 1, 2), workers=_WORKERS)


def spectral_gradient(u, h=1.0):
    """grad u (n2, n1, n0, 3) -> (n2, n1, n0, 3, 3), (grad u)_ij = D_j u_i,
    through the same derivative symbols (full FFT).  Used by the pins."""
    shape = u.shape[:3]
    uh = np.fft.fftn(u, axes=(0, 1, 2))
    D = np.stack(derivative_symbols(shape, h, half=False), axis=-1)
    return np.real(np.fft.ifftn(uh[..., :, None] * D[..., None, :], axes=(0, 1, 2)))
