"""Host-side pieces of the bench: the shock-position report of the blast runs
(bench.shock_radii) and the CPU baseline's sample. Shock radius: on
density fields with a known front, the radius along the 3 axes and 4
diagonals is within one cell of it, centred or across the periodic wrap."""
import math

import numpy as np
import pytest

import bench


def _field(n, fn, center):
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    d = [x - center[0], y - center[1], z - center[2]]
    d = [a - np.round(a) for a in d]                       # periodic distance
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    return fn(r).reshape(-1)


def test_sphere_radius_on_every_ray():
    n = 64
    rho = _field(n, lambda r: 1.0 + 2.0 * (r < 0.23), (0.5, 0.5, 0.5))
    radii = bench.shock_radii(rho, n)
    assert len(radii) == 7
    assert all(abs(r - 0.23) < 1.0 / n for r in radii)


def test_shell_half_maximum_off_centre_across_the_wrap():
    """A Gaussian shell at r = 0.3 (width 0.02, peak 4 over a background of 1):
    the outer half-maximum crossing is at 0.3 + 0.02 sqrt(ln 2)."""
    n = 96
    ctr = (0.15, 0.8, 0.5)
    rho = _field(n, lambda r: 1.0 + 3.0 * np.exp(-((r - 0.3) / 0.02) ** 2), ctr)
    want = 0.3 + 0.02 * math.sqrt(math.log(2.0))
    radii = bench.shock_radii(rho, n, center=ctr)
    assert all(abs(r - want) < 1.0 / n for r in radii)


def test_no_front_inside_half_the_box():
    n = 16
    rho = np.ones(n ** 3)
    rho[0] = 2.0                                           # a peak far from the centre's rays
    assert bench.shock_radii(rho, n) == [None] * 7


def test_cpu_baseline_sample_is_a_physical_run():
    """The oracle's timed sample of the Mach-2 turbulence (an under-resolved
    6^3 box) has negative pressure at face points: without limiters a step
    turns non-finite, with the limiters the plain GPU path also runs (TVB +
    positivity before every stage) it stays finite. The baseline times the
    latter whenever the GPU run limits."""
    import warnings
    cfg = dict(bench.CONFIGS["turb256"], name="turb256")
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        plain = bench.cpu_baseline(cfg, 6, limited=False)
        lim = bench.cpu_baseline(cfg, 6, limited=True)
    assert not np.isfinite(plain["w"]).all()
    assert np.isfinite(lim["w"]).all() and lim["value"] > 0 and lim["cores"] == 1
    assert "positivity" in lim["sample"]


def test_alu_flop_count_of_the_headline_stage():
    """The ALU roofline's flops per cell and stage at degree 2, GLM, 3D (n = 10
    modes, Q_v = 27, Q_f = 9, 9 variables): contractions counted from their
    definitions (2 flop per multiply-add), the pointwise physics as the stated
    estimates (60 per volume point, 500 per face point); the mode counts of
    every (dimension, degree) agree with C(d + D, D)."""
    fl = bench.stage_flops_per_cell(3, 2, "glm", 90)
    V, n, qv, qf, D = 9, 10, 27, 9, 3
    assert fl["projection"] == 2 * V * n * qv == 4_860
    assert fl["volume_integral"] == 2 * V * n * qv * D == 14_580
    assert fl["face_traces"] == 2 * V * n * 2 * D * qf == 9_720          # both sides of the D lower faces
    assert fl["surface_integral"] == 2 * V * n * 2 * D * qf == 9_720
    assert fl["volume_flux_est"] == 60 * qv and fl["hlld_est"] == 500 * D * qf
    assert fl["total"] == 54_000
    for D in (2, 3):
        for d in range(4):
            n = math.comb(d + D, D)
            f = bench.stage_flops_per_cell(D, d, "glm", 9 * n)
            assert f["projection"] == 2 * 9 * n * (d + 1) ** D


def test_hbm_bytes_per_cell_of_the_stage():
    """Algorithmic bytes per cell and stage (each coefficient read once as
    stage input, u^n read in two of three stages, the output written once):
    1,056 B for the 256^3 GLM FP32 form (81 float rows + 9 FP64 means), 896 B
    for the Powell FP32 form at degree 2 (68 + 8), 1,920 B for plain FP64 GLM."""
    assert bench.stage_bytes_per_cell(90, 9) == pytest.approx(1056.0)
    assert bench.stage_bytes_per_cell(76, 8) == pytest.approx(896.0)
    assert bench.stage_bytes_per_cell(90, 9, fp32=False) == pytest.approx(1920.0)


def test_state_l1_closed_form():
    """L1 of eq. lp_norm between two DG states on CPU tensors: a state whose
    density is 2 everywhere against one with density 2.5 + 0.25 xi_x (no sign
    change of the difference): L1_rho = 0.5 / 2 exactly; m_x identical: 0."""
    import numpy as np
    import torch
    from paper_1806_02343_gb300.binding import basis_values
    d, ncell = 2, 40
    g1, gw = np.polynomial.legendre.leggauss(d + 3)
    pts = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    wq = np.einsum("i,j,k->ijk", gw, gw, gw).reshape(-1)
    table = basis_values(3, d, "glm", pts)
    rows = [10 * v for v in range(9)]
    b = torch.zeros((90, 64), dtype=torch.float64)
    b[0, :ncell] = 2.0
    b[10, :ncell] = 1.0
    a = b.clone()
    a[0, :ncell] += 0.5
    a[1, :ncell] = 0.25        # the first degree-1 Legendre mode (xi_x) of rho
    l1 = bench.state_l1(table, a, None, rows, b, None, rows, ncell, wq, chunk=16)
    assert l1[0] == pytest.approx(0.25, rel=1e-13)
    assert l1[1] == 0.0 and all(x == 0.0 for x in l1[2:])


def test_cpu_baseline_all_cores_runs_concurrent_copies():
    cfg = dict(bench.CONFIGS["turb256"], name="turb256")
    r = bench.cpu_baseline_all_cores(cfg, 4, limited=False, procs=2)
    assert r["cores"] == 2 and r["value"] > 0 and r["kind"] == "oracle"
    info = bench.host_info()
    assert info["nproc"] >= 1
