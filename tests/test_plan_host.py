"""The host planner of dynamic regridding (Sec. 5) through the C ABI without a
context or a GPU (dg_mhd_sibling_groups, dg_mhd_regrid_plan_mesh) against the
oracle (oracle/regrid.py: sibling_groups, plan): identical groups, identical
new leaves in Morton order and identical sources, on 2D and 3D meshes with
random refinement and coarsening marks; a hand-checked balance cascade; leaves
given out of Morton order; and the rejection of meshes that are not a 2:1
balanced partition of the cube."""
import itertools

import numpy as np
import pytest

from oracle import regrid as G
from paper_1806_02343_gb300 import workloads as W


@pytest.fixture(scope="module")
def B():
    from paper_1806_02343_gb300 import build, binding
    build.build()
    return binding


def _arrays(leaves):
    lev = np.array([l for l, _ in leaves], dtype=np.int8)
    ijk = np.array([k for _, k in leaves], dtype=np.int32)
    return lev, ijk


def _oracle_arrays(items, D):
    kinds = {"copy": 0, "prolong": 1, "restrict": 2}
    lev = np.array([l for (l, _), _ in items], dtype=np.int8)
    ijk = np.array([k for (_, k), _ in items], dtype=np.int32).reshape(-1, D)
    src = np.array([[kinds[s[0]] | ((s[2] if s[0] == "prolong" else 0) << 4), s[1]] for _, s in items],
                   dtype=np.int32)
    return lev, ijk, src


def _random_marks(leaves, D, seed, p_refine, p_coarsen):
    rng = np.random.default_rng(seed)
    refine = rng.random(len(leaves)) < p_refine
    groups = G.sibling_groups(leaves, D)
    coarsen = [g for g, (_, _, mem) in enumerate(groups) if not refine[mem].any() and rng.random() < p_coarsen]
    marks = np.zeros(len(leaves), dtype=np.int8)
    marks[refine] = 1
    for g in coarsen:
        marks[groups[g][2]] = -1
    return refine, groups, coarsen, marks


def _ball(center, radius):
    return lambda c, dx, l: np.linalg.norm(np.asarray(c) - center) < radius


MESHES = {
    "3d_ball": lambda: W.octree_leaves(3, 1, 4, _ball(0.4, 0.3)),
    "2d_ball": lambda: W.octree_leaves(2, 2, 6, _ball(0.6, 0.25)),
    "2d_uniform": lambda: [(3, k) for k in itertools.product(range(8), repeat=2)],
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_groups_match_oracle(B, name):
    leaves = MESHES[name]()
    D = len(leaves[0][1])
    lev, ijk = _arrays(leaves)
    got = B.sibling_groups(lev, ijk)
    ref = np.array([mem for _, _, mem in G.sibling_groups(leaves, D)], dtype=np.int32).reshape(-1, 2 ** D)
    assert len(ref) > 0 and np.array_equal(got, ref)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_plan_matches_oracle(B, name, seed):
    leaves = MESHES[name]()
    D = len(leaves[0][1])
    refine, groups, coarsen, marks = _random_marks(leaves, D, seed, 0.08, 0.6)
    items = G.plan(leaves, D, refine, groups, coarsen)
    ref = _oracle_arrays(items, D)
    got = B.regrid_plan_mesh(*_arrays(leaves), marks)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["3d_ball", "2d_ball"])
def test_random_marks_exercise_every_rule(B, name):
    """Over the seeds of the parity test: copies, prolongations, restrictions,
    leaves refined only for the balance, and coarsening refused for it."""
    leaves = MESHES[name]()
    D = len(leaves[0][1])
    seen = set()
    for seed in (0, 1, 2):
        refine, _, coarsen, marks = _random_marks(leaves, D, seed, 0.08, 0.6)
        src = B.regrid_plan_mesh(*_arrays(leaves), marks)[2]
        kinds = src[:, 0] & 15
        seen |= {int(k) for k in kinds}
        if any(k & 15 == 1 and not refine[c] for k, c in src):
            seen.add("balance")
        if len(coarsen) > int((kinds == 2).sum()):
            seen.add("refused")
    assert seen == {0, 1, 2, "balance", "refused"}


def test_balance_cascade_by_hand(B):
    """2D, level 2 everywhere except leaf (0,0) split into four level-3 leaves.
    Refining the level-3 leaf (1,1) makes level-4 leaves that touch the level-2
    leaves (1,0) and (0,1), which must split; nothing else changes."""
    leaves = [(3, (0, 0)), (3, (1, 0)), (3, (0, 1)), (3, (1, 1))] + \
             [(2, k) for k in itertools.product(range(4), repeat=2) if k != (0, 0)]
    leaves.sort(key=lambda leaf: G_key(*leaf))
    marks = np.zeros(len(leaves), dtype=np.int8)
    c11 = leaves.index((3, (1, 1)))
    marks[c11] = 1
    lev, ijk, src = B.regrid_plan_mesh(*_arrays(leaves), marks)
    new = {(int(l), tuple(int(x) for x in k)): (int(s[0]), int(s[1])) for l, k, s in zip(lev, ijk, src)}
    for o in range(4):
        assert new[(4, (2 + (o & 1), 2 + (o >> 1)))] == (1 | (o << 4), c11)
    for parent in ((1, 0), (0, 1)):
        old = leaves.index((2, parent))
        for o in range(4):
            assert new[(3, (2 * parent[0] + (o & 1), 2 * parent[1] + (o >> 1)))] == (1 | (o << 4), old)
    assert len(new) == len(leaves) + 3 * 3     # three leaves become four each
    assert (2, (1, 1)) in new and new[(2, (1, 1))][0] == 0


def G_key(l, k, lmax=3):
    """Morton key of the lower corner (axis 0 fastest), then level."""
    z = 0
    kk = [x << (lmax - l) for x in k]
    for bit in range(lmax, -1, -1):
        for a in range(len(k) - 1, -1, -1):
            z = (z << 1) | ((kk[a] >> bit) & 1)
    return (z, l)


def test_leaves_out_of_morton_order(B):
    """The leaves may come in any order: the same new leaves, the sources naming
    the leaves by their given index, the groups by the same numbering."""
    leaves = MESHES["3d_ball"]()
    refine, groups, coarsen, marks = _random_marks(leaves, 3, 7, 0.05, 0.5)
    lev, ijk = _arrays(leaves)
    ref = B.regrid_plan_mesh(lev, ijk, marks)
    perm = np.random.default_rng(3).permutation(len(leaves))
    got = B.regrid_plan_mesh(lev[perm], ijk[perm], marks[perm])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    inv = np.argsort(perm)
    src = got[2].copy()
    leafsrc = (src[:, 0] & 15) != 2
    src[leafsrc, 1] = perm[src[leafsrc, 1]]          # back to the original leaf index
    assert np.array_equal(src, ref[2])
    g_perm = B.sibling_groups(lev[perm], ijk[perm])
    assert np.array_equal(perm[g_perm], B.sibling_groups(lev, ijk))
    assert inv.shape == perm.shape


def test_output_is_a_balanced_partition_and_a_fixed_point(B):
    leaves = MESHES["2d_ball"]()
    _, _, _, marks = _random_marks(leaves, 2, 11, 0.1, 0.5)
    lev, ijk, _ = B.regrid_plan_mesh(*_arrays(leaves), marks)
    B.sibling_groups(lev, ijk)                      # raises unless a balanced partition
    lev2, ijk2, src2 = B.regrid_plan_mesh(lev, ijk, np.zeros(len(lev), dtype=np.int8))
    assert np.array_equal(lev2, lev) and np.array_equal(ijk2, ijk)
    assert np.array_equal(src2[:, 0], np.zeros(len(lev))) and np.array_equal(src2[:, 1], np.arange(len(lev)))


def test_rejects_invalid_meshes_and_marks(B):
    from paper_1806_02343_gb300.binding import DGError
    uni = [(2, k) for k in itertools.product(range(4), repeat=2)]
    lev, ijk = _arrays(uni)
    zero = np.zeros(len(uni), dtype=np.int8)

    def code(lv, kk, mk=None):
        try:
            B.regrid_plan_mesh(lv, kk, zero[: len(lv)] if mk is None else mk)
        except DGError as e:
            return e.code
        return 0

    assert code(lev, ijk) == 0
    assert code(lev[1:], ijk[1:]) == -2                                   # a hole
    assert code(np.append(lev, 1), np.vstack([ijk, [0, 0]]), np.zeros(17, np.int8)) == -2  # overlap
    bad = ijk.copy()
    bad[3] = [4, 0]
    assert code(lev, bad) == -2                                           # coordinate out of range
    # unbalanced: a level-1 leaf next to level-3 leaves
    unb = [(1, (1, 0)), (1, (0, 1)), (1, (1, 1))] + [(2, (1, 0)), (2, (0, 1)), (2, (1, 1))] + \
          [(3, (0, 0)), (3, (1, 0)), (3, (0, 1)), (3, (1, 1))]
    lv, kk = _arrays(unb)
    assert code(lv, kk) == -2
    mk = zero.copy()
    mk[0] = 2
    assert code(lev, ijk, mk) == -1                                       # mark outside {-1, 0, 1}
    assert code(np.full(1, 18, np.int8), np.zeros((1, 2), np.int32), np.zeros(1, np.int8)) == -2


@pytest.mark.parametrize("name", sorted(MESHES) + ["3d_ball_shuffled", "one_leaf"])
def test_octree_faces_match_oracle(B, name):
    """The face list a context builds (dg_mhd_octree_faces) equals the
    oracle's, face by face: left cell, right cell, axis, kind, sub-face."""
    from oracle.amr import AMRScheme
    if name == "3d_ball_shuffled":
        leaves = MESHES["3d_ball"]()
        leaves = [leaves[i] for i in np.random.default_rng(5).permutation(len(leaves))]
    elif name == "one_leaf":
        leaves = [(0, (0, 0, 0))]
    else:
        leaves = MESHES[name]()
    D = len(leaves[0][1])
    A = AMRScheme(D, 1, "glm", 5.0 / 3.0, leaves)
    fl, fr, meta = B.octree_faces(*_arrays(leaves))
    ref = np.array([(cl, cr, a | (kind << 2) | (sub << 4)) for cl, cr, a, kind, sub in A.faces], dtype=np.int32)
    assert len(ref) > 0
    assert np.array_equal(np.stack([fl, fr, meta], 1), ref)
    if name.startswith("3d_ball"):
        assert ((meta >> 2) & 3 == 1).any() and ((meta >> 2) & 3 == 2).any()    # coarse-fine both ways


def test_octree_faces_reject_invalid_meshes(B):
    from paper_1806_02343_gb300.binding import DGError
    uni = [(2, k) for k in itertools.product(range(4), repeat=2)]
    unb = [(1, (1, 0)), (1, (0, 1)), (1, (1, 1))] + [(2, (1, 0)), (2, (0, 1)), (2, (1, 1))] + \
          [(3, (0, 0)), (3, (1, 0)), (3, (0, 1)), (3, (1, 1))]
    for bad in (uni[1:], uni + [(1, (0, 0))], uni + [uni[3]], unb):
        with pytest.raises(DGError) as e:
            B.octree_faces(*_arrays(bad))
        assert e.value.code == -2


def test_orszag_tang_octree_workload(B):
    """The static octree of the Orszag-Tang workload: 1,387,520 leaves of
    levels 5/6/7 (3,072 / 73,728 / 1,310,720) tiling the cube 2:1-balanced
    (the face builder validates it), Morton-sorted, and a z-extrusion: each
    (level, i, j) column holds all 2^level cells along z."""
    lev, ijk = W.orszag_tang_octree()
    assert len(lev) == 1_387_520
    assert np.bincount(lev, minlength=8)[5:8].tolist() == [3_072, 73_728, 1_310_720]
    fl, fr, meta = B.octree_faces(lev, ijk)                   # raises unless a balanced tiling
    assert len(fl) > 3 * len(lev) // 2
    assert ((meta >> 2) & 3).max() > 0                         # coarse-fine faces exist
    cols = {}
    for l, (i, j, k) in zip(lev.tolist(), ijk.tolist()):
        cols.setdefault((l, i, j), set()).add(k)
    assert all(len(ks) == 2 ** l for (l, _, _), ks in cols.items())
    g = B.sibling_groups(lev, ijk)                             # Morton order: groups are index runs
    assert len(g) > 0 and np.all(np.diff(g, axis=1) == 1)


def test_orszag_tang_coarsening_step_of_the_bench(B):
    """The regrid step the octree bench times marks every complete sibling
    group for coarsening (the Orszag-Tang start is smooth at this resolution):
    the 1,387,520 leaves become 204,800 (every one of the 168,960 complete
    groups restricts: 1,387,520 - 7 x 168,960), the counts the bench's GPU
    regrid leg reports, and the new mesh is again a balanced tiling."""
    lev, ijk = W.orszag_tang_octree()
    g = B.sibling_groups(lev, ijk)
    assert len(g) == 168_960
    marks = np.zeros(len(lev), dtype=np.int8)
    marks[g.reshape(-1)] = -1
    lev_n, ijk_n, src = B.regrid_plan_mesh(lev, ijk, marks)
    assert len(lev_n) == 204_800
    assert int(((src[:, 0] & 15) == 2).sum()) == 168_960
    B.octree_faces(lev_n, ijk_n)                              # raises unless a balanced tiling
