"""Parity at the benchmark's full size and launch configuration (256^3,
degree 2, GLM, decaying-turbulence start): one application of the operator on
the GPU, checked on seeded sampled cells against the FP64 oracle evaluated
cell by cell from the same input coefficients. Also the 2D Alfven workload
(32^2, Powell/LDF, 10 SSP-RK3 steps at CFL 0.3) against the oracle and the
closed form, the 64^3 degree-3 workload's FP32 form against its FP64 form, and
the 128^3 degree-2 Powell/LDF blast's operator on sampled cells after three
limited steps (the face jumps of B, and with them the Powell terms, are
non-zero there)."""
import math

import numpy as np
import pytest

from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import from_device, rel_err, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _gather(sol, w, wm, cells, n, mrows=None):
    """Own and face-neighbour weights of sampled cells (FP64 copies of the
    device state; the FP64 means replace the mean rows, by default those of
    the GLM layout)."""
    import torch
    ix, iy, iz = cells % n, (cells // n) % n, cells // (n * n)
    nbrs = []
    for a in range(3):
        for s in (-1, 1):
            jx, jy, jz = ix.copy(), iy.copy(), iz.copy()
            if a == 0: jx = (jx + s) % n
            if a == 1: jy = (jy + s) % n
            if a == 2: jz = (jz + s) % n
            nbrs.append((jz * n + jy) * n + jx)
    allc = np.concatenate([cells] + nbrs)
    idx = torch.as_tensor(allc, device="cuda")
    x = w[:, idx].double().cpu().numpy().T.copy()
    if wm is not None:
        if mrows is None:
            mrows = list(range(0, sol.nrows, sol.nrows // 9))
        x[:, mrows] = wm[:, idx].cpu().numpy().T
    b = len(cells)
    return x[:b], np.stack([x[b * (1 + k): b * (2 + k)] for k in range(6)], 1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_operator_at_full_size_on_sampled_cells(prec):
    import torch
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    n, d = 256, 2
    sol = Solver(3, (n, n, n), d, "glm", precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64)
    w, wm = sol.alloc_state()
    nodal = W.turbulence_nodal(n, d + 1, sol.stride)
    sol.project(nodal, d + 1, w, wm)
    del nodal
    torch.cuda.empty_cache()
    ch, kap = 9.0, 40.0
    sol.set_glm(ch, kap)
    out, om = sol.alloc_state()
    sol.rhs(w, wm, out, om)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2024)
    cells = np.concatenate([rng.choice(n ** 3, 120, replace=False), [0, n - 1, n * n - 1, n ** 3 - 1]])
    S = Scheme(3, d, "glm", G, 4)              # tables only; cell size set below
    S.dx = 1.0 / n
    wc, wnb = _gather(sol, w, wm, cells, n)
    ref = S.rhs_local(wc, wnb, ch, kap)
    got = out[:, torch.as_tensor(cells, device="cuda")].double().cpu().numpy().T
    if prec == "fp64":
        assert rel_err(got, ref) < 1e-12
    else:
        # FP32 operator bound (see the smaller FP32 tests): 2e-4 of the largest
        # value, and the CFL-step update within 1e-6 of the state scale
        assert rel_err(got, ref) < 2e-4
        dt = 0.3 / 5 / (3 * 8.0 * n)
        assert np.max(np.abs(got - ref)) * dt < 1e-6 * np.max(np.abs(wc))
        gm = om[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
        assert rel_err(gm, ref[:, list(range(0, sol.nrows, sol.nrows // 9))]) < 2e-5


def test_alfven_2d_workload_ten_steps():
    import torch
    from paper_1806_02343_gb300.binding import Solver
    S = Scheme(2, 2, "powell", G, 32)
    w0 = S.project(lambda x: W.alfven_2d(x, nvar=8))
    sol = Solver(2, (32, 32), 2, "powell", cfl=0.3)
    w = to_device(w0, sol)
    wo, t = w0.copy(), 0.0
    for _ in range(10):
        sol.step(w)
        wo, dt = S.step(wo)
        t += dt
    got = from_device(w, sol)
    assert rel_err(got, wo) < 1e-11
    err, ref = S.l1_error(got, lambda x: W.alfven_2d(x, t=t, nvar=8))
    assert err[5] / ref[5] < 2e-4        # B_x against the closed form


def test_fourier_64_fp32_form_matches_fp64_form():
    import torch
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    n, d = 64, 3
    F = W.SmoothFourier3D(nvar=9)
    nodal = W.gauss_nodal(F, n, d + 1, 3, ((n ** 3 + 31) // 32) * 32)
    res = {}
    for prec in (DG_PREC_FP64, DG_PREC_FP32MIX):
        sol = Solver(3, (n, n, n), d, "glm", precision=prec)
        w, wm = sol.alloc_state()
        sol.project(nodal, d + 1, w, wm)
        for _ in range(5):
            sol.step(w, wm)
        assert sol.status() == 0
        res[prec] = (w[:, : n ** 3].double(), wm)
    a = res[DG_PREC_FP64][0]
    b = res[DG_PREC_FP32MIX][0]
    # per-variable L2 norm of the field difference: by orthogonality of the basis,
    # ||u||^2 = dx^3 sum_cells sum_l M_l w_l^2 (Sec. 3.1)
    from oracle import basis as OB
    M = torch.as_tensor([float(OB.legendre_mass(k)) for k in OB.mode_list(3, d)], dtype=torch.float64, device="cuda")
    nm = len(M)
    diff = ((a - b) ** 2).reshape(9, nm, -1).sum(2) @ M
    norm = (a ** 2).reshape(9, nm, -1).sum(2) @ M
    rel = torch.sqrt(diff / torch.clamp(norm, min=1e-6 * norm.max())).cpu().numpy()
    assert rel[:8].max() < 1e-5, rel
    # psi starts at zero and is made by the divergence error itself: its
    # difference is measured against the largest variable norm of the run
    assert math.sqrt(diff[8].item() / norm.max().item()) < 1e-5, rel


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_powell_blast_operator_at_full_size_on_sampled_cells(prec):
    import torch
    from gpu_helpers import mean_rows
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64, DG_LIMIT_TVB
    n, d = 128, 2
    sol = Solver(3, (n, n, n), d, "powell", precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64,
                 limiter=DG_LIMIT_TVB, positivity=1)
    w, wm = sol.alloc_state()
    nodal = W.gauss_nodal(lambda x: W.blast_3d(x, nvar=8), n, d + 1, 3, sol.stride, "cuda")
    sol.project(nodal, d + 1, w, wm)
    del nodal
    for _ in range(3):
        sol.step(w, wm)
    out, om = sol.alloc_state()
    sol.rhs(w, wm, out, om)
    torch.cuda.synchronize()
    assert sol.status() == 0
    rng = np.random.default_rng(77)
    # random cells, cells around the blast front (centre 0.5, radius 0.1) and the box corners
    idx = np.arange(n ** 3)
    xc = (np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) + 0.5) / n
    r = np.linalg.norm(xc - 0.5, axis=1)
    front = np.flatnonzero((r > 0.08) & (r < 0.14))
    cells = np.unique(np.concatenate([rng.choice(n ** 3, 100, replace=False), rng.choice(front, 100, replace=False),
                                      [0, n - 1, n * n - 1, n ** 3 - 1]]))
    S = Scheme(3, d, "powell", G, 4)
    S.dx = 1.0 / n
    mr = mean_rows(S)
    wc, wnb = _gather(sol, w, wm, cells, n, mr)
    ref = S.rhs_local(wc, wnb)
    got = out[:, torch.as_tensor(cells, device="cuda")].double().cpu().numpy().T
    # the sampled front cells carry face jumps of B: the Powell terms are exercised
    assert np.max(np.abs(wnb[:, 0, 5 * S.n:] - wc[:, 5 * S.n:])) > 1e-3 * np.max(np.abs(wc[:, 5 * S.n:]))
    if prec == "fp64":
        assert rel_err(got, ref) < 1e-12
    else:
        assert rel_err(got, ref) < 2e-4
        gm = om[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
        assert rel_err(gm, ref[:, mr]) < 2e-5
