"""Solver.project_ic (the initial condition through dg_mhd_project without
depending on the basis ordering) and Solver.eval_at_points against the
oracle's L2 projection and point values: uniform 3D GLM and an octree with
Powell/LDF rows."""
import numpy as np
import pytest

from oracle.amr import AMRScheme
from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import from_device, rel_err

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def test_project_ic_and_eval_uniform_glm():
    from paper_1806_02343_gb300.binding import Solver
    S = Scheme(3, 2, "glm", G, (6, 5, 4))
    fn = W.SmoothFourier3D(nvar=9)
    ref = S.project(fn, npts=5)
    sol = Solver(3, (6, 5, 4), 2, "glm", gamma=G, box_len=S.L)
    w, _ = sol.alloc_state()
    sol.project_ic(fn, w, npts=5)
    assert rel_err(from_device(w, sol), ref) < 1e-12
    pts = np.array([[0.1, -0.3, 0.7], [-1.0, 1.0, 0.0]])
    got = sol.eval_at_points(w, xi=pts).cpu().numpy()                  # [vars, P, cells]
    want = S.eval_points(ref, S.synth(pts))                             # [cells, P, vars]
    assert rel_err(got.transpose(2, 1, 0), want) < 1e-12


def test_project_ic_octree_powell():
    from paper_1806_02343_gb300.binding import Solver
    leaves = W.octree_leaves(3, 2, 3, lambda c, dx, l: np.linalg.norm(np.asarray(c) - 0.5) < 0.3)
    A = AMRScheme(3, 1, "powell", G, leaves)
    fn = W.SmoothFourier3D(nvar=8)
    ref = A.project(fn, npts=4)
    sol = Solver(3, None, 1, "powell", gamma=G, box_len=1.0, leaves=leaves)
    w, _ = sol.alloc_state()
    sol.project_ic(fn, w)
    assert rel_err(from_device(w, sol), ref) < 1e-12
