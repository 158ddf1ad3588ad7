"""Pins of the oracle's spectral operators: rotated-scheme derivative (App. A,
Eq. kas), Nye tensor as curl Fp (App. B) and the Galerkin projection with
mixed control (Sec. 2.2), against closed forms, brute-force DFT sums and the
defining properties of an orthogonal projection onto compatible fields."""
import itertools

import numpy as np

import rvegen
import pytest

from oracle import crystal as cr
from oracle import spectral as sp

UNIAXIAL = np.array([1, 0, 0, 1, 0, 0, 1, 1, 0], dtype=np.uint8)


def grid(shape, h):
    n2, n1, n0 = shape
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    return x * h, y * h, z * h


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_stencil_plane_wave_closed_form(axis):
    # For f = cos(kappa . x): the four-edge difference along e_a at the corner
    # x + h/2 (1,1,1) equals -(2/h) sin(kappa_a h/2) prod_{b != a} cos(kappa_b h/2) sin(kappa . (x + h/2))
    shape, h = (6, 5, 8), 0.37
    kap = 2 * np.pi * np.array([3 / (8 * h), -2 / (5 * h), 1 / (6 * h)])
    x, y, z = grid(shape, h)
    f = np.cos(kap[0] * x + kap[1] * y + kap[2] * z)
    ph = kap[0] * (x + h / 2) + kap[1] * (y + h / 2) + kap[2] * (z + h / 2)
    fac = (2 / h) * np.sin(kap[axis] * h / 2) * np.prod([np.cos(kap[b] * h / 2) for b in range(3) if b != axis])
    assert np.allclose(sp.stencil_derivative(f, axis, h), -fac * np.sin(ph), atol=1e-13)


def test_stencil_matches_spectral_symbol():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((6, 7, 8))
    for a in range(3):
        D = sp.derivative_symbols(f.shape, 0.5, half=False)[a]
        assert np.allclose(np.real(np.fft.ifftn(np.fft.fftn(f) * D)), sp.stencil_derivative(f, a, 0.5), atol=1e-13)


def test_paper_tan_form_equals_symbol_off_nyquist():
    # Eq. kas: k_i = 1/4 tan(xi_i/2) prod_j (1 + e^{i xi_j}); the derivative symbol is i k_i / h
    shape, h = (5, 7, 9), 1.3
    D = sp.derivative_symbols(shape, h, half=False)
    xi = [2 * np.pi * np.fft.fftfreq(n) for n in (9, 7, 5)]
    X0, X1, X2 = xi[0][None, None, :], xi[1][None, :, None], xi[2][:, None, None]
    Z = (1 + np.exp(1j * X0)) * (1 + np.exp(1j * X1)) * (1 + np.exp(1j * X2))
    for a, Xa in enumerate((X0, X1, X2)):
        k = 0.25 * np.tan(Xa / 2) * Z
        assert np.allclose(1j * k / h, D[a], atol=1e-13)


def test_curl_of_discrete_gradient_vanishes():
    # Fp = I + grad u with grad taken by the same derivative: eps_jkl D_k D_l u_i = 0
    rng = np.random.default_rng(2)
    u = rng.standard_normal((6, 6, 8, 3)) * 1e-2
    Fp = np.eye(3) + sp.spectral_gradient(u, 0.7)
    assert np.abs(sp.nye_tensor(Fp, 0.7)).max() < 1e-14


def test_curl_matches_analytic_curl_second_order():
    # Fp_il = delta_il + a_il sin(2 pi x_k(l)/L) with a smooth field; analytic
    # G_ij = -eps_jkl d_k Fp_il at the corner points; error O(h^2)
    L = 1.0
    errs = []
    for n in (8, 16, 32):
        h = L / n
        x, y, z = grid((n, n, n), h)
        xc, yc, zc = x + h / 2, y + h / 2, z + h / 2
        c = 2 * np.pi / L

        def fp(X, Y, Z):
            F = np.zeros(X.shape + (3, 3)); F[..., 0, 0] = F[..., 1, 1] = F[..., 2, 2] = 1
            F[..., 0, 1] += 0.01 * np.sin(c * Z)           # d/dz of Fp_01 -> G_00 = -eps_0 2 1 d_2 Fp_01 = + d_z Fp_01
            F[..., 2, 0] += 0.02 * np.cos(c * Y + c * X)
            F[..., 1, 2] += 0.015 * np.sin(c * X)
            return F
        Fp = fp(x, y, z)
        G = sp.nye_tensor(Fp, h)
        dFp = np.zeros(x.shape + (3, 3, 3))              # [.., i, l, k] = d_k Fp_il at corners
        dFp[..., 0, 1, 2] = 0.01 * c * np.cos(c * zc)
        dFp[..., 2, 0, 0] = -0.02 * c * np.sin(c * yc + c * xc)
        dFp[..., 2, 0, 1] = -0.02 * c * np.sin(c * yc + c * xc)
        dFp[..., 1, 2, 0] = 0.015 * c * np.cos(c * xc)
        Ga = -np.einsum("jkl,...ilk->...ij", sp.LEVI, dFp)
        assert np.abs(Ga[..., 0, 0]).max() > 0.05      # G_00 = + d_z Fp_01 is present
        errs.append(np.abs(G - Ga).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


def test_single_slip_edge_field():
    # Fp = I + gamma(x . s) s (x) m, gamma = g0 sin(kappa . x) with kappa || s:
    # G = -s (x) (grad gamma x m)... evaluated with the stencil gives exactly
    # G_ij = gp * s_i (m x s)_j at the corner, gp = the stencil derivative of gamma
    # along s; A rho18 = vec G and rho18 is the min-norm split.
    s, m = cr.slip_systems()
    a = 2                       # s = [1 -1 0]/sqrt2 on (111): periodic along x and y
    n, h, g0 = 8, 0.5e-6, 1e-3
    x, y, z = grid((n, n, n), h)
    kap = 2 * np.pi / (n * h) * np.array([1.0, -1.0, 0.0])
    gam = g0 * np.sin(kap[0] * x + kap[1] * y)
    Fp = np.eye(3) + gam[..., None, None] * np.outer(s[a], m[a])
    G = sp.nye_tensor(Fp, h)
    ph = kap[0] * (x + h / 2) + kap[1] * (y + h / 2)
    # stencil derivative of gamma along x and y: (2/h) sin(k h/2) cos(k' h/2) cos(0) * cos(phase)
    dgx = g0 * (2 / h) * np.sin(kap[0] * h / 2) * np.cos(kap[1] * h / 2) * np.cos(ph)
    dgy = g0 * (2 / h) * np.sin(kap[1] * h / 2) * np.cos(kap[0] * h / 2) * np.cos(ph)
    grad = np.stack([dgx, dgy, np.zeros_like(dgx)], axis=-1)
    Gexp = -np.einsum("jkl,...k,l,i->...ij", sp.LEVI, grad, m[a], s[a])
    assert np.allclose(G, Gexp, atol=1e-12 * np.abs(Gexp).max())
    # grad gamma || s, so G = |grad| s (x) (m x s): a single edge column of A
    t = np.cross(m[a], s[a])
    gp = grad @ s[a]
    assert np.allclose(G, gp[..., None, None] * np.outer(s[a], t), atol=1e-12 * np.abs(G).max())
    b = 0.256e-9
    A = cr.nye_matrix(np.eye(3), b)
    rho = cr.min_norm_gnd(A, G.reshape(-1, 9).T).T
    assert np.allclose(rho @ A.T, G.reshape(-1, 9), atol=1e-12 * np.abs(G).max())
    # the min-norm split is the projection of the single-edge solution onto row(A),
    # so its norm is below |gp|/b and its active-edge entry is positive
    e = np.zeros(18); e[a] = 1.0
    Pn = np.linalg.pinv(A) @ A
    sel = np.abs(gp.ravel()) > 0.5 * np.abs(gp).max()
    exp = np.outer(gp.ravel()[sel] / b, Pn @ e)
    assert np.allclose(rho[sel], exp, rtol=0, atol=1e-9 * np.abs(exp).max())
    assert np.isclose((Pn @ e)[a], 127.0 / 252.0)     # 0.50397: the active edge keeps about half
    assert np.all(np.linalg.norm(rho[sel], axis=1) < np.abs(gp.ravel()[sel]) / b)


def brute_force_projection(X, mask, h):
    """Pure-loop DFT, projection at every frequency, pure-loop inverse DFT."""
    n2, n1, n0 = X.shape[:3]
    idx = list(itertools.product(range(n2), range(n1), range(n0)))
    out = np.zeros(X.shape, dtype=complex)
    keep = (np.asarray(mask).reshape(3, 3) == 0)
    for (k2, k1, k0) in idx:
        Xh = np.zeros((3, 3), dtype=complex)
        for (z, y, x) in idx:
            Xh += X[z, y, x] * np.exp(-2j * np.pi * (k0 * x / n0 + k1 * y / n1 + k2 * z / n2))
        w = [np.exp(2j * np.pi * k0 / n0), np.exp(2j * np.pi * k1 / n1), np.exp(2j * np.pi * k2 / n2)]
        w = [(-1.0 if (2 * k == n) else wv) for wv, k, n in zip(w, (k0, k1, k2), (n0, n1, n2))]
        D = np.array([(w[0] - 1) * (1 + w[1]) * (1 + w[2]), (1 + w[0]) * (w[1] - 1) * (1 + w[2]),
                      (1 + w[0]) * (1 + w[1]) * (w[2] - 1)]) / (4 * h)
        if k0 == k1 == k2 == 0:
            Gh = np.where(keep, Xh, 0)
        elif np.sum(np.abs(D) ** 2) == 0:
            Gh = np.zeros((3, 3))
        else:
            Gh = np.outer(Xh @ np.conj(D), D) / np.sum(np.abs(D) ** 2)
        for (z, y, x) in idx:
            out[z, y, x] += Gh * np.exp(2j * np.pi * (k0 * x / n0 + k1 * y / n1 + k2 * z / n2))
    return np.real(out) / len(idx)


@pytest.mark.parametrize("shape", [(2, 3, 4), (4, 4, 4), (3, 5, 2)])
def test_projection_brute_force_dft(shape):
    rng = np.random.default_rng(3)
    X = rng.standard_normal(shape + (3, 3))
    assert np.allclose(sp.project(X, UNIAXIAL, 0.3), brute_force_projection(X, UNIAXIAL, 0.3), atol=1e-13)


def test_projection_is_orthogonal_projector_onto_compatible_fields():
    rng = np.random.default_rng(4)
    h = 0.25
    X = rng.standard_normal((6, 4, 8, 3, 3))
    Y = rng.standard_normal((6, 4, 8, 3, 3))
    GX = sp.project(X, UNIAXIAL, h)
    assert np.allclose(sp.project(GX, UNIAXIAL, h), GX, atol=1e-13)            # idempotent
    assert abs(np.sum(GX * Y) - np.sum(X * sp.project(Y, UNIAXIAL, h))) < 1e-11  # self-adjoint
    # compatible: the fluctuation of GX has zero discrete curl (row-wise)
    fl = GX - GX.mean(axis=(0, 1, 2))
    assert np.abs(sp.nye_tensor(fl + np.eye(3), h)).max() < 1e-12
    # the rest is equilibrated: adjoint-stencil divergence sum_j D_j^* (X - GX)_ij = 0
    Rh = np.fft.fftn(X - GX, axes=(0, 1, 2))
    D = np.stack(sp.derivative_symbols(X.shape[:3], h, half=False), -1)
    div = np.einsum("...ij,...j->...i", Rh, np.conj(D))
    assert np.abs(div).max() < 1e-10
    # mean: stress-controlled components kept, strain-controlled ones removed
    keep = (UNIAXIAL.reshape(3, 3) == 0)
    assert np.allclose(GX.mean(axis=(0, 1, 2)), np.where(keep, X.mean(axis=(0, 1, 2)), 0), atol=1e-14)


def test_nyquist_modes_with_two_components_are_zeroed():
    n, h = 4, 1.0
    x, y, z = grid((n, n, n), h)
    X = np.zeros((n, n, n, 3, 3))
    X[..., 0, 1] = np.cos(np.pi * x) * np.cos(np.pi * y)        # xi = (pi, pi, 0): zero symbol
    assert np.abs(sp.project(X, UNIAXIAL, h)).max() < 1e-14
    X[..., 0, 1] = np.cos(np.pi * x)                             # xi = (pi, 0, 0): kept on column 0
    X[..., 0, 0] = np.cos(np.pi * x)
    GX = sp.project(X, UNIAXIAL, h)
    assert np.allclose(GX[..., 0, 0], np.cos(np.pi * x), atol=1e-14)
    assert np.abs(GX[..., 0, 1]).max() < 1e-14


# ---- standard spectral derivative (App. A's continuous frequencies) and the
# Gibbs oscillations it produces at a grain boundary (App. B)

def _band_limited_fp(n, h, seed):
    """Fp = I + sum of three plane waves with |k| below Nyquist on every axis,
    and its exact derivatives d_k Fp_il (analytic)."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    Fp = np.tile(np.eye(3), (n, n, n, 1, 1)).astype(float)
    dFp = np.zeros((n, n, n, 3, 3, 3))
    for _ in range(3):
        kv = rng.integers(-(n // 2 - 1), n // 2, size=3)
        a = 1e-3 * rng.standard_normal((3, 3))
        ph = 2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n + rng.random()
        Fp += a * np.sin(ph)[..., None, None]
        for k in range(3):
            dFp[..., k] += a * (2 * np.pi * kv[k] / (n * h) * np.cos(ph))[..., None, None]
    return Fp, dFp


def test_standard_curl_is_exact_on_band_limited_fields():
    n, h = 12, 0.7
    Fp, dFp = _band_limited_fp(n, h, 5)
    G = sp.nye_tensor_standard(Fp, h)
    exact = -np.einsum("jkl,...ilk->...ij", sp.LEVI, dFp)
    assert np.abs(exact).max() > 1e-3
    assert np.abs(G - exact).max() < 1e-12 * np.abs(exact).max()


def test_standard_curl_of_a_band_limited_gradient_vanishes():
    n, h = 10, 1.3
    rng = np.random.default_rng(9)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    grad = np.zeros((n, n, n, 3, 3))
    for _ in range(4):
        kv = rng.integers(-(n // 2 - 1), n // 2, size=3)
        c = rng.standard_normal(3)
        ph = 2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n
        for j in range(3):           # (grad u)_ij = d_j u_i, u_i = c_i sin(ph)
            grad[..., :, j] += c * (2 * np.pi * kv[j] / (n * h) * np.cos(ph))[..., None]
    G = sp.nye_tensor_standard(np.eye(3) + grad, h)
    assert np.abs(grad).max() > 0.1
    assert np.abs(G).max() < 1e-12 * np.abs(grad).max()


def test_rotated_nye_is_local_and_standard_rings_at_a_slip_jump():
    # App. B: at a jump of Fp the rotated stencil gives a Nye tensor confined to
    # the voxel layers at the boundary; the standard derivative gives Gibbs
    # oscillations that reach into the grains with alternating sign
    n, h = 32, 1.0
    Fp = rvegen.bicrystal_slip_jump(n)
    Gr = np.abs(sp.nye_tensor(Fp, h)).max(axis=(0, 1, 3, 4))      # per x column
    Gs_full = sp.nye_tensor_standard(Fp, h)
    Gs = np.abs(Gs_full).max(axis=(0, 1, 3, 4))
    # the rotated Nye tensor lives on the voxel corners n + 1/2: the jumps
    # between x = 15 | 16 and 31 | 0 land on the layers 15 and 31 alone
    near = [n // 2 - 1, n - 1]
    others = [x for x in range(n) if x not in near]
    assert Gr[near].min() > 1e-5
    assert Gr[others].max() == 0.0                                # exactly local
    centres = [n // 4, 3 * n // 4]
    assert Gs[centres].min() > 0.1 * Gs.max()                     # the ringing reaches the grain centres
    # sign alternation from voxel to voxel along x inside the grains (checkerboard)
    i, j = np.unravel_index(np.abs(Gs_full[0, 0]).max(axis=0).argmax(), (3, 3))
    for grain in (Gs_full[0, 0, : n // 2, i, j], Gs_full[0, 0, n // 2:, i, j]):
        assert np.all(np.sign(grain[1:]) != np.sign(grain[:-1]))
