"""Pins of the regridding oracle (Sec. 5, adaptive mesh refinement): each
check is against something other than the oracle's own matrices --
pointwise evaluation, the L2 definition on a finer rule, closed forms of the
smoothness indicator, and the tiling / 2:1 balance of the new mesh."""
import itertools

import numpy as np
import pytest

from oracle import basis as B
from oracle import mhd
from oracle import regrid as G
from oracle.amr import balanced
from oracle.dg import Scheme

pytestmark = pytest.mark.filterwarnings("ignore")


def _scheme(divb, D=3, d=2):
    return Scheme(D, d, divb, 5.0 / 3.0, 2)


def _random_state(S, rng):
    """Random weights with a divergence-free B (LDF rows are free)."""
    return rng.standard_normal(S.N)


def test_affine_octant_equals_evaluation_at_mapped_points():
    rng = np.random.default_rng(1)
    poly = B.legendre_poly((2, 1, 0))
    poly = B.padd(poly, B.legendre_poly((0, 0, 2)), 3)
    pts = rng.uniform(-1, 1, (50, 3))
    for o in range(8):
        s = np.array(G.octant_sign(o, 3), dtype=float)
        got = B.peval(G.affine_octant(poly, tuple(int(x) for x in s)), pts)
        assert np.allclose(got, B.peval(poly, (pts + s) / 2), atol=1e-14)


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_prolonged_children_reproduce_the_parent_pointwise(divb, D):
    """The parent polynomial (Legendre variables and the LDF B field; in 2D the
    Powell form's B_z Legendre rows too) restricted to octant o is represented
    exactly by child o's weights."""
    S = _scheme(divb, D=D)
    rng = np.random.default_rng(2)
    wp = _random_state(S, rng)
    ch = G.prolong(S, wp)
    pts = rng.uniform(-1, 1, (40, D))
    Sc = S.synth(pts)
    for o in range(2 ** D):
        s = np.array(G.octant_sign(o, D), dtype=float)
        up = np.einsum("r,rqv->qv", wp, S.synth((pts + s) / 2))
        uc = np.einsum("r,rqv->qv", ch[o], Sc)
        assert np.abs(up - uc).max() < 1e-12


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_restriction_is_the_l2_projection_of_the_children(divb, D):
    """Arbitrary children: the residual u_children - u_parent is orthogonal to
    every parent basis row (each octant integrated with its own Gauss rule),
    and the parent mean of every variable is the average of the children's."""
    S = _scheme(divb, D=D)
    rng = np.random.default_rng(3)
    no = 2 ** D
    wc = rng.standard_normal((no, S.N))
    wp = G.restrict(S, wc)
    qp, qw = B.gauss_tensor(D, S.d + 2)
    resid = np.zeros(S.N)
    for o in range(no):
        s = np.array(G.octant_sign(o, D), dtype=float)
        xp = (qp + s) / 2                         # octant points in parent coordinates
        uc = np.einsum("r,rqv->qv", wc[o], S.synth(qp))
        up = np.einsum("r,rqv->qv", wp, S.synth(xp))
        Sp = S.synth(xp)
        resid += np.einsum("qv,rqv,q->r", uc - up, Sp, qw) / no
    assert np.abs(resid).max() < 1e-12
    mp = S.means(wp[None])[0]
    mc = S.means(wc).mean(axis=0)
    assert np.abs(mp - mc).max() < 1e-13


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_restrict_after_prolong_is_identity(divb, D):
    S = _scheme(divb, D=D)
    w = np.random.default_rng(4).standard_normal(S.N)
    assert np.abs(G.restrict(S, G.prolong(S, w)) - w).max() < 1e-13


def _legendre_weights(S, var, poly):
    """Weights of a scalar polynomial in variable `var`'s Legendre rows."""
    w = np.zeros(S.N)
    for r, (kind, v, i) in enumerate(S.rows):
        if kind == "L" and v == var:
            w[r] = float(B.pintegrate(B.pmul(poly, S.legendre[i]))) / S.mass[r]
    return w


def test_smoothness_closed_forms():
    """S_a(xi_a) = 2 * 8 = 16; S_b(xi_a) = 0; S_a(l_2(xi_a)) = 2 int (3 xi)^2 +
    8 int 3^2 = 48 + 576 = 624; S_0(xi_0 xi_1) = 2 int xi_1^2 = 16/3 (3D)."""
    S = _scheme("glm")
    x = {(1, 0, 0): 1}
    s = G.smoothness(S, _legendre_weights(S, mhd.RHO, x)[None], [mhd.RHO])[0, 0]
    assert np.allclose(s, [16.0, 0.0, 0.0], atol=1e-12)
    l2 = {(2, 0, 0): 1.5, (0, 0, 0): -0.5}
    s = G.smoothness(S, _legendre_weights(S, mhd.EN, l2)[None], [mhd.EN])[0, 0]
    assert np.allclose(s, [624.0, 0.0, 0.0], atol=1e-10)
    xy = {(1, 1, 0): 1}
    s = G.smoothness(S, _legendre_weights(S, mhd.RHO, xy)[None], [mhd.RHO])[0, 0]
    assert np.allclose(s, [16.0 / 3.0, 16.0 / 3.0, 0.0], atol=1e-12)


def test_smoothness_of_ldf_b_components():
    """Powell form: B = (xi_1, 0, 0) (divergence-free) from its LDF weights has
    S_1(B_x) = 16 and nothing else."""
    S = _scheme("powell")
    pts, wts = B.gauss_tensor(3, 4)
    Sv = S.synth(pts)
    rows = [r for r, (k, _, _) in enumerate(S.rows) if k == "B"]
    # least squares on the LDF rows for the B components at the points
    A = Sv[rows][:, :, mhd.BX:mhd.BX + 3].reshape(len(rows), -1).T
    target = np.zeros((len(pts), 3))
    target[:, 0] = pts[:, 1]
    coef, *_ = np.linalg.lstsq(A, target.reshape(-1), rcond=None)
    w = np.zeros(S.N)
    w[rows] = coef
    s = G.smoothness(S, w[None], [mhd.BX, mhd.BY, mhd.BZ])[0]
    assert np.allclose(s, [[0, 16, 0], [0, 0, 0], [0, 0, 0]], atol=1e-9)


def _tiles(leaves, D):
    lmax = max(l for l, _ in leaves)
    cover = np.zeros([2 ** lmax] * D, dtype=int)
    for l, k in leaves:
        sl = tuple(slice(x << (lmax - l), (x + 1) << (lmax - l)) for x in k)
        cover[sl] += 1
    return (cover == 1).all()


def _uniform(l, D=3):
    return [(l, k) for k in itertools.product(range(2 ** l), repeat=D)]


def test_plan_refines_balances_and_tiles():
    """Refining one level-2 leaf of a uniform level-1/2 mesh ripples to the
    level-1 neighbours that become two levels coarser; the result tiles the box
    and is 2:1 balanced."""
    leaves = [(1, k) for k in itertools.product(range(2), repeat=3) if k != (0, 0, 0)]
    leaves += [(2, k) for k in itertools.product(range(2), repeat=3)]
    assert balanced(leaves, 3) and _tiles(leaves, 3)
    refine = np.zeros(len(leaves), dtype=bool)
    refine[leaves.index((2, (1, 1, 1)))] = True
    groups = G.sibling_groups(leaves, 3)
    items = G.plan(leaves, 3, refine, groups, [])
    new = [(l, k) for (l, k), _ in items]
    assert _tiles(new, 3) and balanced(new, 3)
    # the level-1 face neighbours of the refined cell were refined too; the
    # level-1 leaf that touches it only along an edge or corner was not
    assert max(l for l, _ in new) == 3
    for k in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        assert (1, k) not in new and (2, tuple(2 * x for x in k)) in new
    assert (1, (1, 1, 1)) in new


def test_plan_coarsens_where_balance_allows():
    """Uniform level-2 mesh: coarsening every group gives the level-1 mesh;
    with one group refined instead, the groups next to it stay fine."""
    leaves = _uniform(2)
    groups = G.sibling_groups(leaves, 3)
    assert len(groups) == 8
    items = G.plan(leaves, 3, np.zeros(len(leaves), bool), groups, list(range(8)))
    assert sorted(l for (l, _), _ in items) == [1] * 8
    refine = np.zeros(len(leaves), bool)
    refine[leaves.index((2, (0, 0, 0)))] = True
    g0 = [g for g, (_, pk, _) in enumerate(groups) if pk == (0, 0, 0)][0]
    items = G.plan(leaves, 3, refine, groups, [g for g in range(8) if g != g0])
    new = [(l, k) for (l, k), _ in items]
    assert _tiles(new, 3) and balanced(new, 3)
    # level-3 cells exist, so no level-1 parent touches them
    assert max(l for l, _ in new) == 3 and (1, (1, 1, 1)) in new


def test_marks_and_remap_keep_totals():
    """A steep tanh profile in rho refines across the front and coarsens the
    flat groups; the remap conserves every variable's total (sum of mean x
    volume)."""
    S = _scheme("glm")
    leaves = _uniform(3)
    h = 0.125
    w = np.zeros((len(leaves), S.N))
    qp, qw = B.gauss_tensor(3, 5)
    Sq = S.synth(qp)
    for c, (l, k) in enumerate(leaves):
        x = (np.array(k) + 0.5 + 0.5 * qp) * h
        u = np.zeros((len(qp), S.V))
        u[:, mhd.RHO] = 1.0 + 0.5 * np.tanh((x[:, 0] - 0.5) / 0.03)
        u[:, mhd.EN] = 2.0
        w[c] = np.einsum("qv,rqv,q->r", u, Sq, qw) / S.mass
    refine, groups, coarsen = G.marks(S, leaves, w, [mhd.RHO], 0.03, 1, 4)
    assert refine.any() and len(coarsen) > 0
    items = G.plan(leaves, 3, refine, groups, coarsen)
    new = [(l, k) for (l, k), _ in items]
    assert _tiles(new, 3) and balanced(new, 3)
    w2 = G.remap(S, w, groups, items)
    vol_old = np.array([8.0 ** -l for l, _ in leaves])
    vol_new = np.array([8.0 ** -l for l, _ in new])
    tot_old = (S.means(w) * vol_old[:, None]).sum(0)
    tot_new = (S.means(w2) * vol_new[:, None]).sum(0)
    assert np.abs(tot_old - tot_new).max() < 1e-13


def test_plan_in_2d_tiles_and_balances():
    """2D quadtree: refining one corner leaf of a level-3 mesh and coarsening
    the groups far from it gives a tiling, 2:1-balanced mesh."""
    leaves = [(3, k) for k in itertools.product(range(8), repeat=2)]
    groups = G.sibling_groups(leaves, 2)
    assert len(groups) == 16
    refine = np.zeros(len(leaves), bool)
    refine[leaves.index((3, (0, 0)))] = True
    far = [g for g, (_, pk, _) in enumerate(groups) if min(pk) >= 2]
    items = G.plan(leaves, 2, refine, groups, far)
    new = [(l, k) for (l, k), _ in items]
    assert _tiles(new, 2) and balanced(new, 2)
    assert sum(1 for l, _ in new if l == 2) == len(far) and sum(1 for l, _ in new if l == 4) == 4
