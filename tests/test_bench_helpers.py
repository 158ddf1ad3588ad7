"""Host logic of bench.py's roofline line (CPU only): which bound a kernel is
rated against, and that the per-launch algorithmic figures follow from the
per-voxel counts."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_fp64_cg_kernels_are_alu_bound_and_fp32_ones_hbm_bound():
    b = bench()
    peaks = {"hbm_gbs": 6789.6}
    shape = (64, 64, 64)
    _, r64 = b.roofline({"tangent_apply": (100, 6.7)}, shape, peaks, prec=0)
    assert r64["bound"] == "alu" and r64["unit"].startswith("GFLOP/s")
    # 81 FMA for K : p, 9 for the p update, 9 for p . t per voxel
    assert r64["algorithmic_flops"] == 64 ** 3 * 198
    _, r32 = b.roofline({"tangent_apply": (100, 2.7)}, shape, peaks, prec=1)
    assert r32["bound"] == "hbm" and r32["unit"] == "GB/s"
    assert r32["algorithmic_bytes"] == r64["algorithmic_bytes"] / 2
    assert abs(r32["achieved"] - r32["algorithmic_bytes"] / 27e-6 / 1e9) < 1e-6 * r32["achieved"]


def test_dominant_kernel_and_share():
    b = bench()
    stats = {"tangent_apply": (10, 0.8), "stencil": (10, 0.5), "constitutive": (0, 0.0)}
    dom, r = b.roofline(stats, (32, 32, 32), {"hbm_gbs": 6789.6})
    assert dom == "tangent_apply" and abs(r["share"] - 0.8 / 1.3) < 1e-12 and r["launches"] == 10


def test_traffic_table_names_known_categories():
    b = bench()
    cats = set(b.kernel_models(64, 64, 64, local=(1, 1, 1)))
    for (cat, prec), v in b.TRAFFIC_64.items():
        assert cat in cats and prec in (0, 1) and v > 0


def test_hall_petch_fit_recovers_known_law():
    # sigma_y = sigma_inf (1 + C (D sqrt(rho))^-x) at four grain sizes
    b = bench()
    import numpy as np
    rho, C, x = 1.0e12, 3.7, 0.66
    d = np.array([62e-6, 40e-6, 27e-6, 17e-6])
    s_inf = np.array([80.0, 81.0, 79.5, 80.4])
    s_y = s_inf * (1 + C * (d * np.sqrt(rho)) ** -x)
    Cf, xf = b.hall_petch_fit(d, s_y, s_inf, rho)
    assert abs(Cf / C - 1) < 1e-12 and abs(xf - x) < 1e-12
    # no strengthening at some size: nothing to fit
    assert b.hall_petch_fit(d, s_inf, s_inf, rho) is None


def test_oracle_slice_takes_the_oracle_mix_exactly():
    # the slice evaluates n_cg / ORACLE_CG_PER_EVAL of the voxels (the last
    # grain cut to size) and times real oracle work
    import rvegen
    m = bench()
    wl = rvegen.WORKLOADS["cu16"]
    n_cg = 6
    secs, nsub, n = m.oracle_slice(wl, n_cg, seed=3)
    assert n == n_cg and secs > 0.0
    assert nsub == round(wl.n ** 3 * n_cg / m.ORACLE_CG_PER_EVAL)
    # a second slice reuses the set-up oracle and picks another subset size-for-size
    secs2, nsub2, _ = m.oracle_slice(wl, n_cg, seed=4)
    assert nsub2 == nsub and secs2 > 0.0


def test_reference_arm_prints_one_line():
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cu16", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
