"""Parity of the CUDA limiters (through dg_mhd_limit / dg_mhd_step) against
the oracle's limiters (Sec. 4.2, 4.3). FP64: 1e-12 relative, identical
troubled-cell flags; FP32 form: 1e-5 relative on the state."""
import numpy as np
import pytest

from oracle import mhd
from oracle.dg import Scheme
from oracle.limiter import Limiter
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import from_device, means_to_device, rel_err, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _shock_field(nvar):
    def fn(x):
        r = np.sqrt((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.55) ** 2)
        inside = r < 0.27
        rho = np.where(inside, 1.0, 0.3)
        p = np.where(inside, 5.0, 0.2)
        one = np.ones_like(rho)
        v = np.stack([0.3 * one, -0.2 * one, 0.1 * one], -1)
        Bv = np.stack([0.8 * one, 0.3 * one, np.where(inside, 0.2, -0.4)], -1)
        u = mhd.conserved(rho, v, p, Bv, G)
        if nvar == 9:
            u = np.concatenate([u, 0.01 * np.sin(6 * x[..., :1])], -1)
        return u
    return fn


def _solver(S, ncell, prec="fp64", **kw):
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    return Solver(S.D, ncell, S.d, S.divb, gamma=G, box_len=S.L,
                  precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64, **kw)


@pytest.mark.parametrize("divb,d,ncell", [("powell", 2, (9, 8, 7)), ("glm", 2, (8, 7, 6)), ("powell", 1, (6, 7, 5))])
def test_tvb_fp64(divb, d, ncell):
    import torch
    S = Scheme(3, d, divb, G, ncell)
    S.P.Mtilde = 0.5
    w0 = S.project(_shock_field(S.V))
    lim = Limiter(S, tvb=True, positivity=False)
    ch = 3.0
    ref, trig = lim.tvb_limit(w0, ch)
    sol = _solver(S, ncell, limiter=1, Mtilde=0.5)
    if divb == "glm":
        sol.set_glm(ch, 1.0)
    w = to_device(w0, sol)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, None, flags)
    got = from_device(w, sol)
    f = flags[: sol.ncell].cpu().numpy().astype(bool)
    assert trig.sum() > 10
    assert np.array_equal(f, trig)
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_positivity_fp64(divb):
    S = Scheme(3, 2, divb, G, (6, 5, 4))
    w0 = S.project(_shock_field(S.V))
    rng = np.random.default_rng(3)
    bad = rng.choice(S.C, 12, replace=False)
    w0[bad, 2] += 0.5                     # rho degree-1 mode
    w0[bad, 4 * S.n + 8] += 4.0           # E degree-2 mode
    lim = Limiter(S, tvb=False, positivity=True)
    ref = lim.positivity(w0)
    sol = _solver(S, (6, 5, 4), positivity=1)
    w = to_device(w0, sol)
    sol.limit(w, None)
    assert rel_err(from_device(w, sol), ref) < 1e-12


@pytest.mark.parametrize("order", [3, 4])
@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_step_with_limiters_fp64(divb, order):
    """Limiters before every stage evaluation (Sec. 4.3), SSP-RK3 and the
    ten-stage fourth-order scheme."""
    S = Scheme(3, 2, divb, G, (8, 7, 6))
    S.P.Mtilde = 0.5
    S.P.rk_order = order
    w0 = S.project(_shock_field(S.V))
    lim = Limiter(S, tvb=True, positivity=True)
    sol = _solver(S, (8, 7, 6), limiter=1, positivity=1, Mtilde=0.5, rk_order=order)
    w = to_device(w0, sol)
    wo = w0.copy()
    for _ in range(2):
        dt = S.dt(lim(wo, None) if divb == "powell" else wo)
        import torch
        dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        sol.step(w, None, dtt)
        ch, kap = S.glm_speeds(dt) if divb == "glm" else (None, 0.0)
        wo, _ = S.step(wo, dt, limiter=lambda x: lim(x, ch))
    assert rel_err(from_device(w, sol), wo) < 1e-10


def test_tvb_fp32_form():
    import torch
    S = Scheme(3, 2, "glm", G, (8, 7, 6))
    S.P.Mtilde = 0.5
    w0 = S.project(_shock_field(S.V))
    lim = Limiter(S, tvb=True, positivity=True)
    ref = lim(w0, 3.0)
    sol = _solver(S, (8, 7, 6), prec="fp32", limiter=1, positivity=1, Mtilde=0.5)
    sol.set_glm(3.0, 1.0)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S)
    sol.limit(w, wm)
    assert rel_err(from_device(w, sol), ref) < 1e-5


@pytest.mark.parametrize("divb,d", [("powell", 2), ("glm", 2), ("powell", 1), ("glm", 1)])
def test_positivity_fp32_form_listed(divb, d):
    """FP32 form, positivity only (Sec. 4.3), 3D degrees 1-2: the FP32 screen
    lists the cells it cannot clear and the listed-cell kernel limits them.
    Planted negative densities and pressures; a few cells below the mean
    floors as well. Result within the FP32 tolerance of the oracle, and the
    counters record the rescaled cells."""
    S = Scheme(3, d, divb, G, (9, 8, 7))
    w0 = S.project(_shock_field(S.V))
    rng = np.random.default_rng(5)
    bad = rng.choice(S.C, 40, replace=False)
    w0[bad, 1] += 0.6 * np.abs(w0[bad, 0])              # rho: degree-1 mode along x
    w0[bad, 4 * S.n + S.n - 1] += 6.0 * np.abs(w0[bad, 4 * S.n])  # E: highest mode
    lim = Limiter(S, tvb=False, positivity=True)
    ref = lim.positivity(w0)
    sol = _solver(S, (9, 8, 7), prec="fp32", positivity=1)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S)
    sol.counters(reset=True)
    sol.limit(w, wm)
    assert sol.counters()["pos_cells"] > 0
    assert rel_err(from_device(w, sol), ref) < 1e-5
