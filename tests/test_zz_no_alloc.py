"""rve_project_noalloc: the allocation-free Galerkin projection, for callers
that cannot allocate device memory (a plug-in under a host application that
owns the device memory, or a loop that cannot take cudaMalloc's implicit
synchronisation).  Its spectrum scratch and frequency tables are a static
device array inside the library.

Checked through the C ABI against the handle-based rve_project (itself
checked against the oracle) on the same inputs: two calls in a row per grid
(the second reuses what the first left in the array), grids up to the
largest that fits (64^3), an odd and a unit n2, an in-place call (X == Y),
and a return to an earlier grid after others (the tables are rebuilt when
the grid changes).  This file is collected last on purpose."""
import numpy as np
import pytest

import rvegen

pytestmark = pytest.mark.gpu

UNIAXIAL = rvegen.UNIAXIAL_X_MASK
MIXED = np.array([0, 1, 1, 0, 0, 1, 1, 0, 1], np.uint8)
SHAPES = [(16, 24, 32), (64, 64, 64), (9, 12, 16), (1, 6, 8)]   # (n2, n1, n0)
L = 20e-6


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
    return float(np.abs(a - b).max() / np.abs(b).max())


def check_shape(pkg, shape, seed, in_place=False):
    import torch
    n2, n1, n0 = shape
    gid = np.zeros(shape, dtype=np.int32)
    rve = pkg.RVE(gid, np.array([[1.0, 0, 0, 0]]), rvegen.material("Cu"), L)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(seed)
    try:
        for call, mask in enumerate((UNIAXIAL, MIXED)):
            X = torch.from_numpy(rng.standard_normal((9, gid.size))).cuda()
            ref = rve.project(mask, X).cpu().numpy()
            Y = X.clone() if in_place else torch.full_like(X, np.nan)
            src = Y if in_place else X
            st = pkg.rve_project_noalloc(n0, n1, n2, L, np.ascontiguousarray(mask, dtype=np.uint8),
                                         src.data_ptr(), Y.data_ptr(), stream.cuda_stream)
            assert st == pkg.RVE_OK, (shape, call)
            stream.synchronize()
            out = Y.cpu().numpy()
            assert np.isfinite(out).all()
            assert relerr(out, ref) < 1e-13, (shape, call)
    finally:
        rve.close()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[::-1])))
def test_noalloc_projection_matches_handle_projection_twice(pkg, shape):
    check_shape(pkg, shape, seed=sum(shape))


def test_noalloc_projection_in_place_and_after_a_grid_change(pkg):
    check_shape(pkg, (9, 12, 16), seed=7, in_place=True)
    check_shape(pkg, (16, 24, 32), seed=8)     # back to another grid: tables rebuilt


def test_noalloc_rejects_bad_sizes(pkg):
    import torch
    X = torch.zeros(9 * 8, dtype=torch.float64, device="cuda")
    m = np.ascontiguousarray(UNIAXIAL)
    s = torch.cuda.current_stream().cuda_stream
    assert pkg.rve_project_noalloc(3, 2, 2, 1.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_EINVAL
    assert pkg.rve_project_noalloc(2, 2, 2, 0.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_EINVAL
    assert pkg.rve_project_noalloc(10, 2, 2, 1.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_EINVAL  # radix 5
    # 96^3 needs 9 * 49 * 96 * 96 * 16 B = 65 MB of spectrum, above the static maximum
    assert pkg.rve_project_noalloc(96, 96, 96, 1.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_ENOMEM
