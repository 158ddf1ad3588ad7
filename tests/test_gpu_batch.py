"""Batched increments (rve_step_batch) and the grain-size effect.

* Handles of different sizes, grain counts and materials stepped together
  (each on its own stream, one host thread per handle) give bit-identical
  fields to the same handles stepped one by one: every reduction is
  deterministic, so concurrency may not change a single bit.
* A failing handle in a batch reports its own status and leaves the others
  and itself usable (atomic steps).
* CG chunks replayed as CUDA graphs are bit-identical to host launches.
* Handles whose launch shapes the autotuner picked give the same increments.
* Size effect (Sec. 3): with the GND density switched off the response does
  not depend on the RVE's physical size at all; with it on, the smaller
  grains harden more."""
import numpy as np
import pytest

import rvegen

pytestmark = pytest.mark.gpu
MASK = rvegen.UNIAXIAL_X_MASK


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


WLS = [rvegen.Workload("b0", 8, 5, "Cu", 0.003, 3, seed=51),
       rvegen.Workload("b1", 12, 9, "Al", 0.003, 3, seed=52),
       rvegen.Workload("b2", 6, 3, "Ag", 0.003, 3, seed=53),
       rvegen.Workload("b3", 16, 12, "Ni", 0.003, 3, seed=54)]


def make(pkg, wl, **kw):
    gid, quat, mat = wl.inputs()
    return pkg.RVE(gid, quat, mat, wl.edge, own_stream=True, **kw)


def test_batch_equals_sequential_bitwise(pkg):
    a = [make(pkg, w) for w in WLS]
    b = [make(pkg, w) for w in WLS]
    for k in range(3):
        infos = pkg.step_batch(a, [w.dFbar() for w in WLS], MASK, np.zeros(9), [w.dt for w in WLS])
        assert all(i["converged"] for i in infos)
        for r, w in zip(b, WLS):
            r.step(w.dFbar(), MASK, np.zeros(9), w.dt)
    for ra, rb in zip(a, b):
        for name in ("F", "P", "FP", "RHO_SSD", "S"):
            assert np.array_equal(ra.field(name), rb.field(name)), name
    for r in a + b:
        r.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cg_graph_replay_is_bit_identical(pkg, precision):
    """rve_options.graphs: chunks of CG iterations replayed as captured CUDA
    graphs give the same bits, the same iteration counts and the same launch
    counts as launching every kernel from the host; profiling events recorded
    inside the graphs give the per-category device times."""
    wl = WLS[3]
    a = make(pkg, wl, graphs=1, precision=precision)
    b = make(pkg, wl, graphs=0, precision=precision)
    a.profile(True)
    b.profile(True)
    for k in range(wl.increments):
        ia = a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        ib = b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert ia["cg_iters"] == ib["cg_iters"] and ia["newton_iters"] == ib["newton_iters"]
    for name in ("F", "P", "FP", "RHO_SSD", "S"):
        assert np.array_equal(a.field(name), b.field(name)), name
    sa, sb = a.kernel_stats(), b.kernel_stats()
    for k in sa:
        assert sa[k][0] == sb[k][0], k
    for k in ("tangent_apply", "stencil", "cg_update", "fft_z_op"):
        assert sa[k][1] > 0, k
    # a second pass with profiling off replays the untimed captures
    a.profile(False)
    a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    assert np.array_equal(a.field("F"), b.field("F"))
    a.close(); b.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_autotuned_handle_matches_default(pkg, precision):
    """rve_options.autotune picks launch shapes from measured times at create;
    the tuned handle converges to the same increments as the default shapes
    (to round-off: the reduction order may differ)."""
    wl = WLS[3]
    a = make(pkg, wl, autotune=1, precision=precision)
    b = make(pkg, wl, precision=precision)
    t = a.tuning()
    assert t["autotuned"] and not b.tuning()["autotuned"]
    assert 0 < t["div_blocks"] <= 4096 and t["fft_fill"] > 0
    for k in range(wl.increments):
        assert a.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
        assert b.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)["converged"]
    for name in ("F", "P", "FP", "RHO_SSD"):
        ra, rb = a.field(name), b.field(name)
        assert np.abs(ra - rb).max() <= 1e-9 * np.abs(rb).max(), name
    a.close(); b.close()


def test_batch_failure_is_per_handle(pkg):
    good = make(pkg, WLS[0])
    bad = make(pkg, WLS[1], max_newton=1)
    F0 = bad.field("F")
    with pytest.raises(pkg.RVEError):
        pkg.step_batch([good, bad], [WLS[0].dFbar(), WLS[1].dFbar()], MASK, np.zeros(9), [WLS[0].dt, WLS[1].dt])
    assert np.array_equal(bad.field("F"), F0)
    assert good.macro_stress()[0][0, 0] > 0          # the good handle committed its increment
    good.close(); bad.close()


def _flow_stress(pkg, L, gnd, n_inc=4):
    wl = rvegen.Workload("hp", 8, 6, "Cu", 0.004, n_inc, seed=61, L=L)
    gid, quat, mat = wl.inputs()
    mat.gnd_enabled = gnd
    r = pkg.RVE(gid, quat, mat, wl.edge)
    for k in range(n_inc):
        r.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
    s = r.macro_stress()[1][0, 0]
    r.close()
    return s


def test_size_effect_only_through_gnd(pkg):
    s_small, s_large = _flow_stress(pkg, 5e-6, False), _flow_stress(pkg, 80e-6, False)
    assert abs(s_small - s_large) < 1e-9 * abs(s_large)
    g_small, g_large = _flow_stress(pkg, 5e-6, True), _flow_stress(pkg, 80e-6, True)
    assert g_small > g_large > s_large * (1 - 1e-9)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_sweep_rve_with_stalling_cg_converges(pkg, precision):
    """Sweep RVE 12 (96^3 voxels, 183 Cu grains): at plastic onset conjugate
    gradients stall on the non-symmetric consistent tangent (solves cut off at
    max_cg, and a direction that no step along lowers the residual); the
    default solver recovers (truncated CG steps, BiCGStab retries) and the
    first two increments converge to the Newton tolerance with the
    strain-controlled means imposed."""
    wl = rvegen.sweep_workloads()[12]
    gid, quat, mat = wl.inputs()
    r = pkg.RVE(gid, quat, mat, wl.edge, precision=precision)
    Fm = np.eye(3)
    for k in range(2):
        info = r.step(wl.dFbar(), MASK, np.zeros(9), wl.dt)
        assert info["converged"], info
        assert info["residual"] <= pkg.DEFAULT_OPTIONS["newton_tol"]
        Fm = Fm + wl.dFbar().reshape(3, 3)
    F = r.field("F").reshape(-1, 3, 3).mean(axis=0)
    m = MASK.reshape(3, 3).astype(bool)
    assert np.abs(F[m] - Fm[m]).max() < 1e-12
    P, _ = r.macro_stress()
    assert np.abs(P[~m]).max() < 1e-6 * abs(P[0, 0])
    r.close()
