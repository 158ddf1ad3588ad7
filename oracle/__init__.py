"""FP64 CPU oracle for one strain increment of FFT-Galerkin homogenisation with
lower-order strain-gradient crystal plasticity (Haouala, Lucarini, LLorca,
Segurado, arXiv:1910.01946).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (no kernels, headers, tables or helpers); both sides
only consume the seeded arrays produced by ``rvegen``.

Everything is plain NumPy in float64, vectorised over voxels, following the
paper's equations in their printed order:

* ``crystal``      slip systems, interaction classes (Table 1), GND segment
                   matrix A (Eq. defA2) and its minimum-norm inverse (Eq. mingnd),
                   rotations and the cubic stiffness (Eq. 4).
* ``spectral``     rotated-scheme derivative (App. A, Eq. kas) in its
                   equivalent real-space stencil form, the Nye tensor as a curl
                   of Fp (App. B), and the Galerkin projection with mixed
                   control (Sec. 2.2, Eqs. weakarbi / eql_discrete2).
* ``constitutive`` the per-voxel implicit crystal-plasticity update (Sec. 2.1,
                   Eqs. 1-9 and Piola) and its consistent tangent.
* ``solver``       one load increment: Nye/GND, hardening, Newton-CG on
                   Eq. linequil2ast, commit of the internal variables.
* ``sensitivity``  forward-mode derivatives of the macroscopic stress curve
                   with respect to (tau0, K, alpha, b) through the same
                   increment equations, pinned by finite differences.

Where the paper is silent, ambiguous or garbled the reading taken is stated
next to the code.  Functions without an independent pin say so.
"""
