"""rve_project_noalloc: the allocation-free Galerkin projection for callers
that cannot allocate device memory (its spectrum scratch is a static device
array inside the library).  Checked through the C ABI against the
handle-based rve_project on the same inputs, on two calls in a row (the
second call reuses the scratch the first one left behind).  This file is
collected last on purpose."""
import numpy as np
import pytest

import rvegen

pytestmark = pytest.mark.gpu

UNIAXIAL = rvegen.UNIAXIAL_X_MASK


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


def test_noalloc_projection_matches_handle_projection_twice(pkg):
    import torch
    shape = (16, 24, 32)                      # (n2, n1, n0)
    n2, n1, n0 = shape
    L = 20e-6
    gid = np.zeros(shape, dtype=np.int32)
    rve = pkg.RVE(gid, np.array([[1.0, 0, 0, 0]]), rvegen.material("Cu"), L)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(123)
    for call, mask in enumerate((UNIAXIAL, np.array([0, 1, 1, 0, 0, 1, 1, 0, 1], np.uint8))):
        X = torch.from_numpy(rng.standard_normal((9, gid.size))).cuda()
        ref = rve.project(mask, X).cpu().numpy()
        Y = torch.full_like(X, np.nan)
        st = pkg.rve_project_noalloc(n0, n1, n2, L, np.ascontiguousarray(mask, dtype=np.uint8),
                                     X.data_ptr(), Y.data_ptr(), stream.cuda_stream)
        assert st == pkg.RVE_OK, call
        stream.synchronize()
        out = Y.cpu().numpy()
        assert np.isfinite(out).all()
        assert relerr(out, ref) < 1e-13, call
    rve.close()


def test_noalloc_rejects_bad_sizes(pkg):
    import torch
    X = torch.zeros(9 * 8, dtype=torch.float64, device="cuda")
    m = np.ascontiguousarray(UNIAXIAL)
    s = torch.cuda.current_stream().cuda_stream
    assert pkg.rve_project_noalloc(3, 2, 2, 1.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_EINVAL
    assert pkg.rve_project_noalloc(2, 2, 2, 0.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_EINVAL
    # 96^3 needs 9 * 49 * 96 * 96 * 16 B = 65 MB of spectrum, above the static maximum
    assert pkg.rve_project_noalloc(96, 96, 96, 1.0, m, X.data_ptr(), X.data_ptr(), s) == pkg.RVE_ENOMEM
