"""Pins of the oracle on static octree meshes (Sec. 4.4): no GPU."""
import numpy as np
import pytest

from oracle.amr import AMRScheme, balanced
from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

G = 5.0 / 3.0


def _sphere_mesh(D=3, lo=2, hi=4, r=0.3):
    return W.octree_leaves(D, lo, hi, lambda c, dx, l: np.linalg.norm(c - 0.5) < r)


def test_octree_generator_is_balanced_and_covers_the_box():
    for D in (2, 3):
        leaves = _sphere_mesh(D)
        assert balanced(leaves, D)
        vol = sum(2.0 ** (-D * l) for l, _ in leaves)
        assert abs(vol - 1.0) < 1e-15
        assert len({l for l, _ in leaves}) >= 3


@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_uniform_octree_equals_uniform_scheme(divb):
    leaves = W.octree_leaves(3, 2, 2, lambda c, dx, l: False)
    A = AMRScheme(3, 2, divb, G, leaves)
    U = Scheme(3, 2, divb, G, 4)
    perm = [(k[2] * 4 + k[1]) * 4 + k[0] for _, k in leaves]
    fn = W.SmoothFourier3D(nvar=A.V)
    wa, wu = A.project(fn), U.project(fn)
    assert np.array_equal(wa, wu[perm])
    assert np.max(np.abs(A.rhs(wa, 2.0, 1.0) - U.rhs(wu, 2.0, 1.0)[perm])) < 1e-14 * np.abs(U.rhs(wu, 2.0, 1.0)).max()


@pytest.mark.parametrize("D,divb", [(3, "glm"), (3, "powell"), (2, "powell"), (2, "glm")])
def test_amr_free_stream_and_conservation(D, divb):
    leaves = _sphere_mesh(D)
    A = AMRScheme(D, 2, divb, G, leaves)
    assert any(f[3] > 0 for f in A.faces)        # coarse-fine faces present
    w = A.project(lambda x: W.uniform_state(x, nvar=A.V))
    assert np.max(np.abs(A.rhs(w, 2.0, 0.5))) < 1e-12
    fn = W.SmoothFourier3D(nvar=A.V) if D == 3 else (lambda x: W.alfven_2d(x, nvar=A.V))
    w = A.project(fn)
    r = A.rhs(w, 3.0, 0.0)
    tot = A.totals(r)
    scale = np.abs(A.means(r)).max()
    if divb == "glm":
        assert np.max(np.abs(tot)) < 1e-13 * scale
    else:
        assert abs(tot[0]) < 1e-13 * scale


def test_amr_alfven_2d_static_refinement_converges():
    # the 2D Alfven wave on meshes with a refined band keeps order ~3
    errs = []
    for lo in (3, 4):
        leaves = W.octree_leaves(2, lo, lo + 1, lambda c, dx, l: abs(c[0] - 0.5) < 0.2)
        A = AMRScheme(2, 2, "powell", G, leaves)
        w = A.project(lambda x: W.alfven_2d(x, nvar=8))
        t, T = 0.0, 0.03
        while t < T - 1e-14:
            dt = min(A.dt(w), T - t)
            w, _ = A.step(w, dt)
            t += dt
        e, _ = A.l1_error(w, lambda x: W.alfven_2d(x, t=t, nvar=8))
        errs.append(e[5])
    order = np.log2(errs[0] / errs[1])
    assert 2.5 < order < 3.7, order


def test_amr_mean_differences_reduce_to_uniform():
    from oracle.limiter import Limiter
    leaves = W.octree_leaves(3, 2, 2, lambda c, dx, l: False)
    A = AMRScheme(3, 2, "powell", G, leaves)
    U = Scheme(3, 2, "powell", G, 4)
    perm = [(k[2] * 4 + k[1]) * 4 + k[0] for _, k in leaves]
    fn = W.SmoothFourier3D(nvar=8)
    wa, wu = A.project(fn), U.project(fn)
    da = Limiter(A).mean_differences(A.means(wa))
    du = Limiter(U).mean_differences(U.means(wu))
    assert np.allclose(da[0], du[0][perm], atol=1e-15) and np.allclose(da[1], du[1][perm], atol=1e-15)


def test_amr_mean_differences_exact_for_linear_field():
    # a linear field has D+ = D- = slope along the axis (in reference units) at
    # every cell, whatever the neighbour levels (distance-weighted differences)
    from oracle.limiter import Limiter
    from oracle import mhd
    leaves = W.octree_leaves(3, 2, 3, lambda c, dx, l: c[0] < 0.5)
    A = AMRScheme(3, 1, "powell", G, leaves)
    m = np.zeros((A.C, 8))
    m[:, 0] = 1.0 + 0.3 * A.centers[:, 0]
    dp, dm = Limiter(A).mean_differences(m)
    ix = A.centers[:, 0]
    inner = (ix > 0.2) & (ix < 0.8)          # away from the periodic wrap in x
    expect = 0.3 * A.dxc / 2
    assert np.allclose(dp[inner, 0, 0], expect[inner], atol=1e-14)
    assert np.allclose(dm[inner, 0, 0], expect[inner], atol=1e-14)
