"""Pins of the oracle's crystallography, elasticity and GND algebra (Sec. 2.1,
Tables 1-2, Eqs. defA, defA2, mingnd) against closed forms, published values
and library routines that the oracle itself does not use."""
import json
import os

import numpy as np
import pytest

import rvegen
from oracle import crystal as cr

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_vector():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    r = rvegen.SplitMix64(g["seed"])
    assert [r.next_u64() for _ in range(len(g["first"]))] == g["first"]


def test_quaternions_uniform_rotations():
    q = rvegen.random_quaternions(4000, 99)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-15)
    R = np.array([cr.rotation(x) for x in q])
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-14)
    # Haar measure on SO(3): E[R] = 0, E[R_ij^2] = 1/3
    assert np.abs(R.mean(axis=0)).max() < 4.0 / np.sqrt(4000)
    assert np.abs((R ** 2).mean(axis=0) - 1.0 / 3.0).max() < 0.03


def test_voronoi_periodic_and_tie_break():
    gid, seeds = rvegen.voronoi_grain_map(8, 5, 3)
    assert gid.shape == (8, 8, 8) and gid.dtype == np.int32
    # brute force of one voxel with explicit periodic images
    z, y, x = 5, 2, 7
    c = (np.array([x, y, z]) + 0.5) / 8
    best = min(range(5), key=lambda g: (min(np.sum((c - seeds[g] - np.array(o)) ** 2)
                                            for o in np.ndindex(3, 3, 3) for o in [np.array(o) - 1]), g))
    assert gid[z, y, x] == best
    # two seeds mirror-symmetric about x = 1/2: voxel columns split evenly
    g2, _ = rvegen.voronoi_grain_map(4, 2, 0)
    assert set(np.unique(g2)) <= {0, 1}


def test_slip_systems_geometry():
    s, m = cr.slip_systems()
    assert np.allclose(np.linalg.norm(s, axis=1), 1) and np.allclose(np.linalg.norm(m, axis=1), 1)
    assert np.allclose(np.sum(s * m, axis=1), 0.0, atol=1e-15)
    for a in range(12):
        for b in range(a + 1, 12):
            assert not (np.allclose(m[a], m[b]) and np.isclose(abs(s[a] @ s[b]), 1.0))
    # each <110> direction lies in exactly two {111} planes
    counts = np.array([np.sum(np.abs(np.abs(s @ d) - 1) < 1e-12) for d in cr.SCREW_DIRS])
    assert (counts == 2).all()


def test_interaction_classes_counts_and_symmetry():
    cls = cr.interaction_classes()
    assert (cls == cls.T).all()
    for a in range(12):
        assert [int((cls[a] == k).sum()) for k in range(6)] == [1, 2, 1, 2, 4, 2]
    t1 = json.load(open(os.path.join(GOLD, "paper_tables.json")))["table1"]
    q6 = [t1[k] for k in ("q_self", "q_coplanar", "q_collinear", "q_hirth", "q_glissile", "q_lomer")]
    assert tuple(q6) == rvegen.Q_TABLE1
    q = cr.interaction_matrix(q6, normalise=False)
    assert np.isclose(q.sum(axis=1), 0.122 + 2 * 0.122 + 0.657 + 2 * 0.084 + 4 * 0.137 + 2 * 0.118).all()
    assert np.allclose(np.diag(cr.interaction_matrix(q6)), 1.0)


def test_glissile_vs_lomer_textbook_pair():
    # Planes (111) and (-1 1 1) meet along [0 1 -1].  With b1 = [0 1 -1] (along the
    # intersection) and b2 = [1 0 1]: b1 + b2 = [1 1 0] lies in (-1 1 1): glissile.
    # With b1 = [-1 0 1] and b2 = [1 1 0] (neither along it): b1 + b2 = [0 1 1]
    # lies in neither plane: Lomer-Cottrell lock.  Perpendicular b: Hirth lock.
    s, m = cr.slip_systems()
    cls = cr.interaction_classes()

    def idx(plane, d):
        for a in range(12):
            if np.allclose(m[a], np.array(plane) / np.sqrt(3)) and np.isclose(abs(s[a] @ np.array(d)) / np.sqrt(2), 1.0):
                return a
        raise KeyError
    assert cls[idx([1, 1, 1], [0, 1, -1]), idx([-1, 1, 1], [1, 0, 1])] == 4
    assert cls[idx([1, 1, 1], [-1, 0, 1]), idx([-1, 1, 1], [1, 1, 0])] == 5
    assert cls[idx([1, 1, 1], [0, 1, -1]), idx([1, -1, 1], [0, 1, 1])] == 3
    assert cls[idx([1, 1, 1], [0, 1, -1]), idx([-1, 1, 1], [0, 1, -1])] == 2
    assert cls[idx([1, 1, 1], [0, 1, -1]), idx([1, 1, 1], [1, -1, 0])] == 1


def test_shear_modulus_reproduces_table2():
    t2 = json.load(open(os.path.join(GOLD, "paper_tables.json")))["table2"]
    for name, row in t2.items():
        mu = cr.shear_modulus(row["C11"], row["C12"], row["C44"])
        # Table 2 prints mu to three figures; Al's printed 25.0 is 1.1 % above the
        # value its own C11, C12, C44 give (24.72), the other three agree to 0.05 GPa
        tol = 0.3 if name == "Al" else 0.06
        assert abs(mu - row["mu"]) < tol, (name, mu)


def test_cubic_stiffness_symmetries():
    C = cr.cubic_stiffness(168.4, 121.4, 75.4)
    assert np.allclose(C, np.transpose(C, (1, 0, 2, 3))) and np.allclose(C, np.transpose(C, (2, 3, 0, 1)))
    # a cube symmetry (90 deg about z) leaves it unchanged; a general rotation keeps
    # the isotropic invariants C_iijj and C_ijij
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    assert np.allclose(cr.rotate4(C, Rz), C)
    R = cr.rotation(rvegen.random_quaternions(1, 4)[0])
    Cr = cr.rotate4(C, R)
    assert np.isclose(np.einsum("iijj", Cr), np.einsum("iijj", C))
    assert np.isclose(np.einsum("ijij", Cr), np.einsum("ijij", C))
    # textbook entries: C_1111 = C11, C_1122 = C12, C_1212 = C44
    assert np.allclose([C[0, 0, 0, 0], C[0, 0, 1, 1], C[0, 1, 0, 1], C[0, 0, 0, 1]], [168.4, 121.4, 75.4, 0.0])


def test_nye_matrix_rank_and_min_norm_inverse():
    rng = np.random.default_rng(5)
    R = cr.rotation(rvegen.random_quaternions(1, 8)[0])
    A = cr.nye_matrix(R, 0.256e-9)
    assert A.shape == (9, 18) and np.linalg.matrix_rank(A) == 9
    An = cr.nye_matrix(np.eye(3), 1.0)
    ev = np.linalg.eigvalsh(An @ An.T)
    assert np.isclose(ev.max() / ev.min(), 14.0 / 9.0)
    G = rng.standard_normal((9, 5)) * 1e6
    rho = cr.min_norm_gnd(A, G)
    assert np.allclose(A @ rho, G, rtol=0, atol=1e-14 * np.abs(G).max())
    # equals the SVD minimum-norm solution and is orthogonal to null(A)
    assert np.allclose(rho, np.linalg.pinv(A) @ G, rtol=1e-10, atol=1e-10 * np.abs(rho).max())
    null = np.linalg.svd(A)[2][9:]
    assert np.abs(null @ rho).max() < 1e-10 * np.abs(rho).max()


def test_rotated_frame_gnd_equals_crystal_frame():
    # rho from the sample-frame A equals rho from the crystal-frame A applied to R^T G R
    R = cr.rotation(rvegen.random_quaternions(1, 2)[0])
    G = np.random.default_rng(0).standard_normal((3, 3))
    r1 = cr.min_norm_gnd(cr.nye_matrix(R, 1.0), G.reshape(9))
    r2 = cr.min_norm_gnd(cr.nye_matrix(np.eye(3), 1.0), (R.T @ G @ R).reshape(9))
    assert np.allclose(r1, r2, atol=1e-13)
