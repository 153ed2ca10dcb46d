"""The library's host basis generator (Legendre products and the LDF basis of
Sec. 3.2-3.3 / App. A.2, built in double precision) through the context-free
C ABI dg_mhd_basis_values, against the oracle's exact-rational basis
(Scheme.synth): every state row's field at reference points, for 2D and 3D,
degrees 0-3, both schemes. Also the mean-row list and point evaluation of the
binding (eval_points) against the oracle's eval_points. CPU only."""
import itertools

import numpy as np
import pytest

from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

G = 5.0 / 3.0


@pytest.fixture(scope="module")
def B():
    from paper_1806_02343_gb300 import build, binding
    build.build()
    return binding


def _points(D, seed=0):
    rng = np.random.default_rng(seed)
    corners = np.array(list(itertools.product((-1.0, 1.0), repeat=D)))
    return np.vstack([rng.uniform(-1, 1, (17, D)), corners, np.zeros((1, D))])


CASES = [(D, d, divb) for D in (2, 3) for d in range(4) for divb in ("glm", "powell")]


@pytest.mark.parametrize("D,d,divb", CASES)
def test_basis_values_match_oracle(B, D, d, divb):
    S = Scheme(D, d, divb, G, 2)
    pts = _points(D, seed=d)
    got = B.basis_values(D, d, divb, pts)                 # [rows, vars, P]
    ref = S.synth(pts).transpose(0, 2, 1)                 # [rows, vars, P]
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("D,d,divb", CASES)
def test_mean_rows_are_the_degree_zero_rows(B, D, d, divb):
    S = Scheme(D, d, divb, G, 2)
    assert B.mean_rows(D, d, divb, S.N) == np.flatnonzero(S.is_mean).tolist()


@pytest.mark.parametrize("divb", ["glm", "powell"])
def test_eval_points_matches_oracle(B, divb):
    import torch
    S = Scheme(3, 2, divb, G, (3, 3, 2))
    w0 = S.project(W.SmoothFourier3D(nvar=S.V))
    pts = _points(3, seed=7)
    ref = S.eval_points(w0, S.synth(pts))                 # [cells, P, vars]
    table = B.basis_values(3, 2, divb, pts)
    got = B.eval_points(table, torch.as_tensor(w0.T.copy())).numpy()   # [vars, P, cells]
    assert np.abs(got.transpose(2, 1, 0) - ref).max() <= 1e-13 * np.abs(ref).max()
    # FP32 rows with the FP64 means put back: exact where only the means are non-zero
    rows = B.mean_rows(3, 2, divb, S.N)
    wmean_only = np.zeros_like(w0)
    wmean_only[:, rows] = w0[:, rows]
    w32 = torch.as_tensor(wmean_only.T.copy()).float()
    got32 = B.eval_points(table, w32, rows, torch.as_tensor(w0[:, rows].T.copy())).numpy()
    ref_m = S.eval_points(wmean_only, S.synth(pts))
    assert np.abs(got32.transpose(2, 1, 0) - ref_m).max() <= 1e-15 * np.abs(ref_m).max()


def test_basis_values_rejects_bad_arguments(B):
    from paper_1806_02343_gb300.binding import DGError
    for args in ((4, 2, "glm"), (3, 4, "glm"), (2, -1, "powell")):
        with pytest.raises(DGError) as e:
            B.basis_values(args[0], args[1], args[2], np.zeros((1, args[0])))
        assert e.value.code == -1


def test_cell_points_match_oracle_geometry(B):
    """The Gauss points project_ic evaluates at: cell centre + dx/2 * tensor
    Gauss nodes (last axis fastest), cells in mesh order, for uniform boxes
    (cells per axis unequal, 2D and 3D) and an octree."""
    from oracle import basis as OB
    from oracle.amr import AMRScheme
    for D, ncell, npts in ((3, (4, 3, 2), 3), (2, (5, 3), 4)):
        S = Scheme(D, 1, "glm", G, ncell)
        qp, _ = OB.gauss_tensor(D, npts)
        ref = S.centers[:, None, :] + 0.5 * S.dx * qp[None, :, :]
        got = B.cell_points(D, npts, S.L, n=ncell).numpy()
        assert got.shape == ref.shape and np.abs(got - ref).max() < 1e-14
    leaves = W.octree_leaves(3, 1, 3, lambda c, dx, l: np.linalg.norm(np.asarray(c) - 0.3) < 0.25)
    A = AMRScheme(3, 1, "powell", G, leaves)
    qp, _ = OB.gauss_tensor(3, 2)
    ref = A.centers[:, None, :] + 0.5 * A.dxc[:, None, None] * qp[None, :, :]
    lev = [l for l, _ in leaves]
    ijk = [k for _, k in leaves]
    got = B.cell_points(3, 2, 1.0, levels=lev, ijk=ijk).numpy()
    assert np.abs(got - ref).max() < 1e-14


def _full(S, blockL, blockB):
    """Block-diagonal matrix over the scheme's rows from per-basis blocks."""
    M = np.zeros((S.N, S.N))
    for r1, (k1, v1, i1) in enumerate(S.rows):
        for r2, (k2, v2, i2) in enumerate(S.rows):
            if k1 == k2 == "L" and v1 == v2:
                M[r1, r2] = blockL[i1, i2]
            elif k1 == k2 == "B":
                M[r1, r2] = blockB[i1, i2]
    return M


@pytest.mark.parametrize("D,d,divb", [c for c in CASES if c[1] >= 1])
def test_regrid_tables_match_oracle(B, D, d, divb):
    """dg_mhd_regrid_tables (the host tables of the regridding kernels) against
    the oracle: prolongation and restriction matrices of every octant, and the
    smoothness indicator as quadratic forms on random weights (Sec. 5)."""
    from oracle import mhd
    from oracle import regrid as RG
    S = Scheme(D, d, divb, G, 2)
    T = B.regrid_tables(D, d, divb)
    Pr, Re = RG.prolongation(S), RG.restriction(S)
    for o in range(2 ** D):
        assert np.abs(_full(S, T["PL"][o], T["PB"][o]) - Pr[o]).max() < 1e-12
        assert np.abs(_full(S, T["RL"][o], T["RB"][o]) - Re[o]).max() < 1e-12
    rng = np.random.default_rng(d + 10 * D)
    w = rng.standard_normal((5, S.N))
    fields = (mhd.RHO, mhd.BX, mhd.BY, mhd.BZ)
    ref = RG.smoothness(S, w, fields)                      # [cells, fields, D]
    for fi, v in enumerate(fields):
        legrows = [(r, i) for r, (k, vv, i) in enumerate(S.rows) if k == "L" and vv == v]
        for a in range(D):
            if legrows:
                idx = [r for r, _ in legrows]
                modes = [i for _, i in legrows]
                got = np.einsum("cl,lm,cm->c", w[:, idx], T["QL"][a][np.ix_(modes, modes)], w[:, idx])
            else:                                          # a component of the LDF field
                brow = [(r, i) for r, (k, _, i) in enumerate(S.rows) if k == "B"]
                idx = [r for r, _ in brow]
                js = [i for _, i in brow]
                c = v - mhd.BX
                got = np.einsum("cj,jm,cm->c", w[:, idx], T["QB"][c, a][np.ix_(js, js)], w[:, idx])
            assert np.abs(got - ref[:, fi, a]).max() <= 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("case", ["uniform", "octree"])
def test_project_ic_input_preparation(B, case):
    """project_ic's host side without a GPU: with dg_mhd_project replaced by a
    capture, the point values it hands over, projected with the oracle's own
    formula (sum_q w_q u phi / M), give the oracle's L2 projection."""
    import types
    import torch
    from oracle import basis as OB
    from oracle.amr import AMRScheme
    obj = types.SimpleNamespace()
    if case == "uniform":
        S = Scheme(3, 2, "glm", G, (6, 5, 4))
        fn, npts = W.SmoothFourier3D(nvar=9), 5
        obj.dim, obj.degree, obj.box_len, obj._n, obj._lev, obj._ijk = 3, 2, S.L, [6, 5, 4], None, None
        obj.ncell = obj.stride = 120
    else:
        leaves = W.octree_leaves(3, 2, 3, lambda c, dx, l: np.linalg.norm(np.asarray(c) - 0.5) < 0.3)
        S = AMRScheme(3, 1, "powell", G, leaves)
        fn, npts = W.SmoothFourier3D(nvar=8), None
        obj.dim, obj.degree, obj.box_len, obj._n = 3, 1, 1.0, None
        obj._lev = np.array([l for l, _ in leaves], dtype=np.int8)
        obj._ijk = np.array([k for _, k in leaves], dtype=np.int32).reshape(-1)
        obj.ncell, obj.stride = len(leaves), (len(leaves) + 3) // 4 * 4
    seen = {}
    obj.project = lambda nodal, q, w, wmean=None: seen.update(nodal=nodal, q=q)
    B.Solver.project_ic(obj, fn, torch.zeros((S.N, obj.stride), dtype=torch.float64), npts=npts)
    q = seen["q"]
    assert q == (npts or min(8, obj.degree + 3))
    qp, qw = OB.gauss_tensor(3, q)
    u = seen["nodal"][:, :, : obj.ncell].permute(2, 1, 0).numpy()
    mine = np.einsum("cqv,q,rqv->cr", u, qw, S.synth(qp)) / S.mass
    assert np.abs(mine - S.project(fn, npts=q)).max() < 1e-14
    assert torch.all(seen["nodal"][:, :, obj.ncell:] == 0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_ldf_legendre_map_matches_oracle(d):
    """The map with which the specialised Powell kernels carry B in the Legendre
    form of its components (LDF coefficients mapped on load, residuals mapped
    back on store) equals the oracle's exact rational projection of every LDF
    function onto the Legendre modes, and has the structure the kernels rely
    on: three constant functions, each along one axis, and no other function
    with a non-zero mean."""
    from oracle import mlp as M
    from oracle.dg import Scheme
    from paper_1806_02343_gb300 import binding
    S = Scheme(3, d, "powell", 5.0 / 3.0, (2, 2, 2))
    ref = M.ldf_to_legendre(S)
    A = binding.ldf_legendre(d)
    assert A.shape == ref.shape
    assert np.max(np.abs(A - ref)) < 1e-13
    assert np.all(A[:3, :, 1:] == 0.0)
    axes = [np.flatnonzero(A[j, :, 0]) for j in range(3)]
    assert all(len(x) == 1 for x in axes) and sorted(int(x[0]) for x in axes) == [0, 1, 2]
    assert np.all(A[3:, :, 0] == 0.0)
