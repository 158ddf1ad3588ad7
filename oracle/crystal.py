"""FCC crystallography and elasticity for the oracle (test infrastructure only).

Sec. 2.1 of the paper: 12 {111}<110> slip systems (Eq. 2), the Taylor
interaction matrix built from the six interaction classes of Table 1
(Eq. Taylor_hard), the 18 GND segments (12 edge + 6 screw) and the Nye
matrix A with G = A rho (Eqs. defA, defA2), the minimum-norm GND densities
(Eq. mingnd), and the cubic stiffness tensor (Eq. 4) rotated to the sample frame.
"""
from __future__ import annotations

import numpy as np

_PLANES = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.float64)
_DIRS = {
    0: [[0, 1, -1], [-1, 0, 1], [1, -1, 0]],
    1: [[0, 1, -1], [1, 0, 1], [1, 1, 0]],
    2: [[0, 1, 1], [1, 0, -1], [1, 1, 0]],
    3: [[0, 1, 1], [1, 0, 1], [1, -1, 0]],
}
# the six <110> line directions of the screw GND segments
SCREW_DIRS = np.array([[0, 1, -1], [1, 0, -1], [1, -1, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]],
                      dtype=np.float64) / np.sqrt(2.0)

CLASS_NAMES = ("self", "coplanar", "collinear", "hirth", "glissile", "lomer")


def slip_systems():
    """(s, m): unit slip directions and plane normals of the 12 FCC systems,
    crystal frame, shape (12, 3) each.  Eq. 2: Lp = sum_a gdot^a s^a (x) m^a."""
    s, m = [], []
    for p in range(4):
        for d in _DIRS[p]:
            s.append(np.array(d, dtype=np.float64) / np.sqrt(2.0))
            m.append(_PLANES[p] / np.sqrt(3.0))
    return np.array(s), np.array(m)


def interaction_classes():
    """12x12 integer class index (into CLASS_NAMES) for each pair of systems.

    The paper lists the six coefficients (Table 1) but not the pair layout;
    the classes follow from geometry: same system -> self; same plane ->
    coplanar; parallel Burgers vectors -> collinear; perpendicular Burgers
    vectors -> Hirth lock; otherwise the junction Burgers vector b_a -/+ b_b
    (a <110> vector) lies in one of the two slip planes -> glissile junction,
    else -> Lomer-Cottrell lock.
    """
    s, m = slip_systems()
    cls = np.zeros((12, 12), dtype=np.int64)
    for a in range(12):
        for b in range(12):
            sb = s[a] @ s[b]
            if a == b:
                c = 0
            elif abs(abs(m[a] @ m[b]) - 1.0) < 1e-12:
                c = 1
            elif abs(abs(sb) - 1.0) < 1e-12:
                c = 2
            elif abs(sb) < 1e-12:
                c = 3
            else:
                bj = s[a] - np.sign(sb) * s[b]
                in_a = abs(bj @ m[a]) < 1e-12
                in_b = abs(bj @ m[b]) < 1e-12
                c = 4 if (in_a or in_b) else 5
            cls[a, b] = c
    return cls


def interaction_matrix(q6, normalise: bool = True):
    """q^{ab} of Eq. Taylor_hard from the six Table-1 coefficients.  With
    normalise=True the matrix is divided by the self coefficient (the Taylor
    coefficient alpha then carries the magnitude)."""
    q6 = np.asarray(q6, dtype=np.float64)
    q = q6[interaction_classes()]
    return q / q6[0] if normalise else q


def gnd_segments():
    """Unit Burgers vectors and unit line directions of the 18 GND segments
    (12 edge: b = s, t = m x s; 6 screw: b = t = <110>), crystal frame."""
    s, m = slip_systems()
    b_edge, t_edge = s, np.cross(m, s)
    return (np.concatenate([b_edge, SCREW_DIRS]), np.concatenate([t_edge, SCREW_DIRS]))


def screw_of_system():
    """Index (0..5) of the screw direction parallel to each system's slip direction."""
    s, _ = slip_systems()
    return np.array([int(np.argmax(np.abs(SCREW_DIRS @ s[a]))) for a in range(12)])


def nye_matrix(R, burgers):
    """A (9 x 18) of Eq. defA2 in the sample frame: column a = vec(b b^a (x) t^a),
    row-major vec (index 3i+j), for rotation R (crystal -> sample)."""
    bv, tv = gnd_segments()
    bs, ts = bv @ R.T, tv @ R.T
    return burgers * np.einsum("ai,aj->ija", bs, ts).reshape(9, 18)


def min_norm_gnd(A, g9):
    """Eq. mingnd: the L2-minimal rho with A rho = G.  The printed closed form
    (A^T A)^{-1} A^T is singular for a 9 x 18 matrix; the minimiser of
    rho^T rho subject to A rho = G is A^T (A A^T)^{-1} G, used here."""
    return A.T @ np.linalg.solve(A @ A.T, g9)


def rotation(quat):
    """Rotation matrix (crystal -> sample) of a unit quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(quat, dtype=np.float64) / np.linalg.norm(quat)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def cubic_stiffness(C11, C12, C44):
    """Fourth-order cubic stiffness C_pqrs in the crystal frame (Eq. 4)."""
    d = np.eye(3)
    C = (C12 * np.einsum("pq,rs->pqrs", d, d)
         + C44 * (np.einsum("pr,qs->pqrs", d, d) + np.einsum("ps,qr->pqrs", d, d)))
    for a in range(3):
        C[a, a, a, a] += C11 - C12 - 2 * C44
    return C


def rotate4(C, R):
    """C_ijkl = R_ip R_jq R_kr R_ls C_pqrs."""
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", R, R, R, R, C)


def shear_modulus(C11, C12, C44):
    """Shear modulus for <110>{111} shear of a cubic crystal (Table 2, row mu):
    mu = 3 C44 (C11 - C12) / (4 C44 + C11 - C12)."""
    return 3.0 * C44 * (C11 - C12) / (4.0 * C44 + C11 - C12)
