"""Parity of the Powell face term with q^dagger of eq. powellq-interp (Sec.
4.1.3; dg_mhd_params.powell_q = 1) against the oracle, on uniform meshes
(degrees 1 and 2, FP64 and the FP32 form) and on an octree with coarse-fine
faces. The states carry random higher modes so that B^n jumps at every face
and the choice of q^dagger changes the rhs by far more than the tolerance."""
import numpy as np
import pytest

from oracle.amr import AMRScheme
from oracle.dg import Params, Scheme
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import from_device, means_to_device, rel_err, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _rough(S, w0, seed):
    """Random higher modes (5% of each row's scale): jumps of B^n at the faces."""
    rng = np.random.default_rng(seed)
    w = w0.copy()
    nonmean = ~S.is_mean
    scale = np.abs(w0).max(axis=0, keepdims=True) + 1e-3
    w[:, nonmean] += 0.05 * (scale * rng.standard_normal(w.shape))[:, nonmean]
    return w


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-4)])
@pytest.mark.parametrize("d", [1, 2])
def test_rhs_interp_q_matches_oracle(d, prec, tol):
    import torch
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    ncell = (5, 6, 7)
    S = Scheme(3, d, "powell", G, ncell, params=Params(powell_q="interp"))
    w0 = _rough(S, S.project(W.SmoothFourier3D(nvar=8)), 10 + d)
    ref = S.rhs(w0)
    ref_mean = Scheme(3, d, "powell", G, ncell).rhs(w0)
    assert rel_err(ref_mean, ref) > 50 * tol   # the choice of q^dagger matters here
    sol = Solver(3, ncell, d, "powell", gamma=G, box_len=S.L, powell_q=1,
                 precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64)
    w = to_device(w0, sol)
    out = torch.full_like(w, float("nan"))
    if prec == "fp32":
        wm = means_to_device(w0, sol, S)
        om = torch.full_like(wm, float("nan"))
        sol.rhs(w, wm, out, om)
    else:
        sol.rhs(w, None, out)
    assert rel_err(from_device(out, sol), ref) < tol


def test_rhs_interp_q_matches_oracle_octree():
    import torch
    from paper_1806_02343_gb300.binding import Solver
    leaves = W.octree_leaves(3, 2, 4, lambda c, dx, l: np.linalg.norm(c - 0.45) < 0.3)
    A = AMRScheme(3, 2, "powell", G, leaves, params=Params(powell_q="interp"))
    w0 = _rough(A, A.project(W.SmoothFourier3D(nvar=8)), 7)
    ref = A.rhs(w0)
    ref_mean = AMRScheme(3, 2, "powell", G, leaves).rhs(w0)
    assert rel_err(ref_mean, ref) > 1e-8
    sol = Solver(3, None, 2, "powell", gamma=G, box_len=1.0, leaves=leaves, powell_q=1)
    w = to_device(w0, sol)
    out = torch.full_like(w, float("nan"))
    sol.rhs(w, None, out)
    assert rel_err(from_device(out, sol), ref) < 1e-12
