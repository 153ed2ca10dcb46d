"""Parity of dynamic regridding (Sec. 5, adaptive mesh refinement) through the
C ABI against the oracle (oracle/regrid.py): the smoothness indicator, the
refinement marks, the new leaf list with its sources, and the remapped state
(prolongation / restriction). FP64: 1e-11 relative; FP32 form: 1e-6 relative
on the state (the means remap in FP64)."""
import itertools

import numpy as np
import pytest

from oracle import mhd
from oracle import regrid as G
from oracle.amr import AMRScheme

from gpu_helpers import from_device, means_to_device, rel_err, to_device

pytestmark = pytest.mark.gpu
GAM = 5.0 / 3.0
FIELDS = (mhd.RHO, mhd.BX, mhd.BY, mhd.BZ)


def _front(nvar):
    """A steep front along x (tanh, width 0.03) in the density and in B_y
    (divergence-free); flat elsewhere."""
    def fn(x):
        rho = 1.0 + 0.5 * np.tanh((x[..., 0] - 0.47) / 0.03)
        one = np.ones_like(rho)
        v = np.stack([0.2 * one, 0.1 * one, 0.0 * one], -1)
        p = 1.0 * one
        Bv = np.stack([0.5 * one, 0.2 * np.tanh((x[..., 0] - 0.47) / 0.03), 0.1 * one], -1)
        u = mhd.conserved(rho, v, p, Bv, GAM)
        if nvar == 9:
            u = np.concatenate([u, 0.0 * one[..., None]], -1)
        return u
    return fn


def _leaves(l=3):
    return [(l, k) for k in itertools.product(range(2 ** l), repeat=3)]


def _solver(divb, prec, leaves):
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    kw = {"c_h_fixed": 3.0} if divb == "glm" else {}   # octree GLM: a global c_h
    return Solver(3, None, 2, divb, gamma=GAM, box_len=1.0, leaves=leaves,
                  precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64, **kw)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_smoothness_matches_oracle(divb, prec):
    leaves = _leaves(2)
    A = AMRScheme(3, 2, divb, GAM, leaves)
    w0 = A.project(_front(A.V))
    ref = G.smoothness(A, w0, FIELDS).reshape(len(leaves), -1).max(axis=1)
    sol = _solver(divb, prec, leaves)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A) if prec == "fp32" else None
    got = sol.smoothness(w, wm, FIELDS).cpu().numpy()
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert np.abs(got - ref).max() <= tol * ref.max()
    assert ref.max() > 1.0 and ref.min() < 1e-6  # the front and the flat cells


def _oracle_plan(A, leaves, w0, s_tilde, lo, hi):
    refine, groups, coarsen = G.marks(A, leaves, w0, FIELDS, s_tilde, lo, hi)
    items = G.plan(leaves, 3, refine, groups, coarsen)
    marks = np.zeros(len(leaves), dtype=np.int8)
    marks[refine] = 1
    for g in coarsen:
        marks[groups[g][2]] = -1
    return marks, groups, items


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_marks_plan_and_remap_match_oracle(divb, prec):
    leaves = _leaves(3)
    A = AMRScheme(3, 2, divb, GAM, leaves)
    w0 = A.project(_front(A.V))
    s_tilde, lo, hi = 0.03, 2, 5
    marks_ref, groups, items = _oracle_plan(A, leaves, w0, s_tilde, lo, hi)
    assert (marks_ref == 1).any() and (marks_ref == -1).any()
    sol = _solver(divb, prec, leaves)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A) if prec == "fp32" else None
    marks, _ = sol.amr_marks(w, wm, FIELDS, s_tilde, lo, hi)
    assert np.array_equal(marks.cpu().numpy(), marks_ref)
    lev, ijk, src = sol.regrid_plan(marks)
    assert [(int(l), tuple(int(x) for x in k)) for l, k in zip(lev, ijk)] == [key for key, _ in items]
    kinds = {"copy": 0, "prolong": 1, "restrict": 2}
    src_ref = np.array([[kinds[s[0]] | ((s[2] if s[0] == "prolong" else 0) << 4), s[1]] for _, s in items])
    assert np.array_equal(src, src_ref)
    new, wn, wmn = sol.regrid(w, wm, marks=marks)
    ref = G.remap(A, w0, groups, items)
    got = from_device(wn, new)
    if prec == "fp32":
        got_means = wmn[:, : new.ncell].cpu().numpy().T
        # a prolonged child's mean includes the parent's higher modes, which the
        # FP32 form holds in FP32: a few ulp of FP32 times |slope| / |mean|
        assert rel_err(got_means, ref[:, [r for r in range(A.N) if A.is_mean[r]]]) < 1e-7
        assert rel_err(got, ref) < 1e-6
    else:
        assert rel_err(got, ref) < 1e-11
    assert new.status(1) == 0


@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_regridded_state_conserves_totals_and_steps(divb):
    """The remap keeps every variable's total (sum of mean x cell volume); the
    new context then advances with a finite state."""
    import torch
    leaves = _leaves(3)
    A = AMRScheme(3, 2, divb, GAM, leaves)
    w0 = A.project(_front(A.V))
    sol = _solver(divb, "fp64", leaves)
    w = to_device(w0, sol)
    marks, _ = sol.amr_marks(w, None, FIELDS, 0.03, 2, 5)
    lev_new, _, _ = sol.regrid_plan(marks)
    new, wn, _ = sol.regrid(w, None, marks=marks)
    assert new.ncell == len(lev_new) != sol.ncell
    lev = np.array([l for l, _ in leaves], dtype=float)
    got = from_device(wn, new)
    tot_old = (A.means(w0) * (8.0 ** -lev)[:, None]).sum(0)
    tot_new = (A.means(got) * (8.0 ** -lev_new.astype(float))[:, None]).sum(0)
    assert np.abs(tot_old - tot_new).max() < 1e-12
    new.step(wn, None)
    torch.cuda.synchronize()
    assert new.status(1) in (0, 1)
    assert torch.isfinite(wn[:, : new.ncell]).all()


def test_remap_rejects_out_of_range_sources():
    """Source entries out of range are skipped on the device and reported as
    DG_E_ARG by the new context's status word."""
    import torch
    from paper_1806_02343_gb300 import binding as Bd
    leaves = _leaves(2)
    sol = _solver("glm", "fp64", leaves)
    new = _solver("glm", "fp64", leaves)
    w, _ = sol.alloc_state()
    wn, _ = new.alloc_state()
    src = torch.zeros((new.ncell, 2), dtype=torch.int32, device="cuda")
    src[:, 1] = torch.arange(new.ncell, dtype=torch.int32, device="cuda")
    src[5, 1] = sol.ncell + 7                  # an old cell that does not exist
    src[9, 0] = 2                              # restriction of a group that does not exist
    src[9, 1] = 1 << 20
    rc = Bd.lib().dg_mhd_remap(sol.h, new.h, Bd._ptr(src), Bd._ptr(w), None, Bd._ptr(wn), None, Bd._stream())
    assert rc == 0
    assert new.status(1) == -1  # DG_E_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_marks_plan_and_remap_match_oracle_2d(divb, prec):
    """The same on a 2D quadtree (level 4, 256 leaves): groups of four, the
    2D Powell form's B_z Legendre rows next to its LDF rows."""
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    leaves = [(4, k) for k in itertools.product(range(16), repeat=2)]
    A = AMRScheme(2, 2, divb, GAM, leaves)
    w0 = A.project(_front(A.V))
    s_tilde, lo, hi = 0.03, 3, 6
    refine, groups, coarsen = G.marks(A, leaves, w0, FIELDS, s_tilde, lo, hi)
    items = G.plan(leaves, 2, refine, groups, coarsen)
    marks_ref = np.zeros(len(leaves), dtype=np.int8)
    marks_ref[refine] = 1
    for g in coarsen:
        marks_ref[groups[g][2]] = -1
    assert (marks_ref == 1).any() and (marks_ref == -1).any()
    kw = {"c_h_fixed": 3.0} if divb == "glm" else {}
    sol = Solver(2, None, 2, divb, gamma=GAM, box_len=1.0, leaves=leaves,
                 precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64, **kw)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A) if prec == "fp32" else None
    marks, _ = sol.amr_marks(w, wm, FIELDS, s_tilde, lo, hi)
    assert np.array_equal(marks.cpu().numpy(), marks_ref)
    lev, ijk, src = sol.regrid_plan(marks)
    assert [(int(l), tuple(int(x) for x in k)) for l, k in zip(lev, ijk)] == [key for key, _ in items]
    new, wn, wmn = sol.regrid(w, wm, marks=marks)
    ref = G.remap(A, w0, groups, items)
    assert rel_err(from_device(wn, new), ref) < (1e-6 if prec == "fp32" else 1e-11)
    assert new.status(True) == 0


def test_smoothness_on_a_uniform_mesh():
    """dg_mhd_smoothness takes uniform meshes too (FP64, Powell, 6 x 5 x 4)."""
    from oracle.dg import Scheme
    from paper_1806_02343_gb300.binding import Solver
    S = Scheme(3, 2, "powell", GAM, (6, 5, 4))
    w0 = S.project(_front(S.V))
    ref = G.smoothness(S, w0, FIELDS).reshape(S.C, -1).max(axis=1)
    sol = Solver(3, (6, 5, 4), 2, "powell", gamma=GAM, box_len=S.L)
    got = sol.smoothness(to_device(w0, sol), None, FIELDS).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-11 * ref.max()


def test_regrid_cycles_in_the_time_loop_match_oracle():
    """Regridding inside the time loop (paper_1806_02343_gb300/evolve.py): five
    SSP-RK3 steps of the FP64 Powell scheme (degree 1) from the steep front on
    a level-3 octree, regridding before steps 2 and 4 (marks on rho and B,
    S~ = 0.03, levels 2..5), against the oracle doing the same with its own
    marks, plan, remap and steps: the same leaves after every cycle, the state
    to 1e-11, both refinements and coarsenings among the cycles."""
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP64
    from paper_1806_02343_gb300.evolve import evolve_amr
    leaves = _leaves(3)
    d, s_tilde, lo, hi, steps, every = 1, 0.03, 2, 4, 5, 2
    A = AMRScheme(3, d, "powell", GAM, leaves)
    w0 = A.project(_front(A.V))
    # oracle: the same loop
    w, lv = w0.copy(), list(leaves)
    n_ref = n_coarse = 0
    meshes = []
    for n in range(steps):
        if n > 0 and n % every == 0:
            refine, groups, coarsen = G.marks(A, lv, w, FIELDS, s_tilde, lo, hi)
            n_ref += int(refine.sum())
            n_coarse += len(coarsen)
            items = G.plan(lv, 3, refine, groups, coarsen)
            w = G.remap(A, w, groups, items)
            lv = [key for key, _ in items]
            A = AMRScheme(3, d, "powell", GAM, lv)
            meshes.append(len(lv))
        w, _ = A.step(w)
    assert n_ref > 0 and n_coarse > 0
    sol = Solver(3, None, d, "powell", gamma=GAM, box_len=1.0, leaves=leaves, precision=DG_PREC_FP64)
    sol, wg, _, hist = evolve_amr(sol, to_device(w0, sol), None, steps, every, FIELDS, s_tilde, lo, hi)
    assert [h["cells_after"] for h in hist] == meshes
    assert sum(h["refined"] for h in hist) == n_ref and sum(h["coarsened_groups"] for h in hist) == n_coarse
    got_leaves = [(int(l), tuple(int(x) for x in k)) for l, k in zip(sol._lev, sol._ijk.reshape(-1, 3))]
    assert got_leaves == lv
    assert rel_err(from_device(wg, sol), w) < 1e-11
    assert sol.status(1) == 0
