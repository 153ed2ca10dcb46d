"""Pins of the oracle's limiters (Sec. 4.2, 4.3) -- no GPU."""
import numpy as np
import pytest

from oracle import mhd
from oracle.dg import Scheme
from oracle.limiter import Limiter, eigensystem, dU_dW, dW_dU

G = 5.0 / 3.0


def _jac_fd(f, U, h=1e-6):
    n = len(U)
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h * max(1.0, abs(U[k]))
        J[:, k] = (f(U + e) - f(U - e)) / (2 * e[k])
    return J


STATES = [
    (1.3, (0.4, -0.7, 0.2), 0.8, (0.6, 0.3, -0.5)),
    (0.7, (-1.1, 0.2, 0.5), 2.0, (1.5, 0.0, 0.0)),      # B_t = 0 (alpha / beta degeneracy)
    (1.0, (0.3, 0.1, -0.2), 0.5, (0.0, 0.8, 0.4)),       # B_n = 0
    (2.0, (0.0, 0.0, 0.0), 1.0, (0.0, 0.0, 0.0)),       # no field
]


@pytest.mark.parametrize("st", STATES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_powell_eigensystem_diagonalises_8wave_jacobian(st, axis):
    rho, v, p, Bv = st
    U = mhd.conserved(np.array(rho), np.array(v), np.array(p), np.array(Bv), G)
    R, L, lam = eigensystem(U, axis, G)
    assert np.allclose(L @ R, np.eye(8), atol=1e-10)
    # Powell system: du/dt + (df/du + q e_Bn^T) du/dx = 0 (eq. powell-src in 1D)
    A = _jac_fd(lambda x: mhd.flux(x, axis, G), U)
    A[:, mhd.BX + axis] += mhd.powell_q(U, G)
    assert np.allclose(R @ np.diag(lam) @ L, A, atol=1e-6 * max(1.0, np.abs(A).max()))


@pytest.mark.parametrize("st", STATES[:3])
@pytest.mark.parametrize("axis", [0, 2])
def test_glm_eigensystem(st, axis):
    rho, v, p, Bv = st
    ch = 4.0
    U = mhd.conserved(np.array(rho), np.array(v), np.array(p), np.array(Bv), G, psi=np.array(0.3))
    R, L, lam = eigensystem(U, axis, G, ch)
    assert np.allclose(L @ R, np.eye(9), atol=1e-10)
    # the MHD waves are those of the Powell-form system; the (B_n, psi) pair
    # is the linear GLM subsystem dB_n/dt + dpsi/dx = 0, dpsi/dt + c_h^2 dB_n/dx = 0
    A8 = _jac_fd(lambda x: mhd.flux(x, axis, G), U[:8])
    A8[:, mhd.BX + axis] += mhd.powell_q(U[:8], G)
    AW = dW_dU(U, G)[:8, :8] @ A8 @ dU_dW(U, G)[:8, :8]
    W9 = np.zeros((9, 9))
    W9[:8, :8] = AW
    b = mhd.BX + axis
    W9[b, :] = 0.0
    W9[:, b] = 0.0
    W9[b, 8] = 1.0
    W9[8, b] = ch * ch
    A = dU_dW(U, G) @ W9 @ dW_dU(U, G)
    assert np.allclose(R @ np.diag(lam) @ L, A, atol=1e-6 * max(1.0, np.abs(A).max()))
    assert np.isclose(sorted(lam)[0], -ch) and np.isclose(sorted(lam)[-1], ch)


def _linear_field(x, nvar=8):
    rho = 1.0 + 0.05 * x[..., 0]
    one = np.ones_like(rho)
    return mhd.conserved(rho, np.stack([0.1 * one, 0 * one, 0 * one], -1), one,
                         np.stack([0.5 * one, 0.2 * one, 0 * one], -1), G)


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_tvb_not_triggered_on_linear_data_and_keeps_means(divb):
    S = Scheme(3, 2, divb, G, (12, 3, 3))
    nv = S.V
    fn = lambda x: np.concatenate([_linear_field(x), np.zeros(x.shape[:-1] + (nv - 8,))], -1)
    w = S.project(fn)
    lim = Limiter(S, tvb=True, positivity=False)
    out, troubled = lim.tvb_limit(w, ch=3.0)
    ix = np.arange(S.C) % 12
    interior = (ix > 0) & (ix < 11)
    assert not troubled[interior].any()
    assert np.allclose(S.means(out), S.means(w), atol=1e-14)
    # slopes below M~ dx are never limited (Sec. 4.2.1); with M~ = 0 the
    # periodic wrap -- a jump -- is limited while linear data still is not
    S.P.Mtilde = 0.0
    out, troubled = lim.tvb_limit(w, ch=3.0)
    assert not troubled[interior].any()
    assert troubled[~interior].any()


def _step_field(x, nvar=8):
    rho = np.where(x[..., 0] < 0.47, 1.0, 0.125)   # jump inside cell 7 of 16
    p = np.where(x[..., 0] < 0.47, 1.0, 0.1)
    one = np.ones_like(rho)
    u = mhd.conserved(rho, np.stack([0 * one, 0 * one, 0 * one], -1), p,
                      np.stack([0.75 * one, 1.0 * one, 0 * one], -1), G)
    if nvar == 9:
        u = np.concatenate([u, np.zeros(u.shape[:-1] + (1,))], -1)
    return u


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_tvb_limits_a_jump_conservatively(divb):
    S = Scheme(3, 2, divb, G, (16, 2, 2))
    w = S.project(lambda x: _step_field(x, S.V))
    S.P.Mtilde = 0.5
    lim = Limiter(S, tvb=True, positivity=False)
    out, troubled = lim.tvb_limit(w, ch=3.0)
    ix = np.arange(S.C) % 16
    assert troubled[ix == 7].all()
    assert not troubled[(ix > 0) & (ix < 15) & (np.abs(ix - 7) > 1)].any()
    assert np.allclose(S.means(out), S.means(w), atol=1e-14)
    # limited cells: every weight of degree >= 2 is zero
    deg = np.array([sum(S.modes[i]) if k == "L" else (lim.ldf_deg[i] if k == "B" else 0)
                    for k, v, i in S.rows])
    assert np.all(out[troubled][:, deg >= 2] == 0.0)
    # the limited density slope along x lies within the TVD bounds of the means
    m = S.means(out)
    sl = lim.slopes(out)
    for c in np.where(troubled)[0]:
        cp, cm = S.nbr_plus[0][c], S.nbr_minus[0][c]
        lo = min(m[cp, 0], m[cm, 0], m[c, 0])
        hi = max(m[cp, 0], m[cm, 0], m[c, 0])
        for s in (-1, 1):
            val = m[c, 0] + s * sl[c, 0, 0]
            assert lo - 1e-12 <= val <= hi + 1e-12


def test_ldf_fix_is_divergence_free_and_diminishing():
    S = Scheme(3, 2, "powell", G, (4, 4, 4))
    lim = Limiter(S)
    rng = np.random.default_rng(5)
    out = np.zeros((1, S.N))
    mean = np.zeros(8)
    mean[mhd.BX:mhd.BX + 3] = [0.3, -0.2, 0.5]
    sl = rng.normal(size=(3, 8))           # divergent limited slopes: diag sum != 0
    lim._assign(out, 0, mean, sl)
    got = lim.slopes(out)[0]
    diag = np.array([got[a, mhd.BX + a] for a in range(3)])
    orig = np.array([sl[a, mhd.BX + a] for a in range(3)])
    assert abs(diag.sum()) < 1e-13
    assert np.all(np.abs(diag) <= np.abs(orig) + 1e-14)
    # off-diagonal slopes are untouched; cell mean of B is the given mean
    for a in range(3):
        for c in range(3):
            if a != c:
                assert abs(got[a, mhd.BX + c] - sl[a, mhd.BX + c]) < 1e-13
    assert np.allclose(S.means(out)[0, mhd.BX:mhd.BX + 3], mean[mhd.BX:mhd.BX + 3], atol=1e-14)


def test_positivity_limiter():
    S = Scheme(3, 2, "glm", G, (3, 3, 3))
    rng = np.random.default_rng(7)
    w = S.project(lambda x: np.concatenate([mhd.conserved(np.ones(x.shape[:-1]), np.zeros(x.shape[:-1] + (3,)),
                                                          np.ones(x.shape[:-1]), 0.3 * np.ones(x.shape[:-1] + (3,)),
                                                          G), np.zeros(x.shape[:-1] + (1,))], -1))
    # strong high-order perturbations of rho and E in some cells
    bad = [0, 5, 13]
    w[bad, 4] += 0.8          # a degree-1 rho mode
    w[bad, 4 * S.n + 7] += 3.0  # a degree-2 E mode
    lim = Limiter(S, tvb=False, positivity=True)
    out = lim.positivity(w)
    u = np.einsum("cr,rqv->cqv", out, lim.Spos)
    rho, v, p, _ = mhd.primitives(u, G)
    assert rho.min() >= S.P.eps_rho - 1e-15 and p.min() >= S.P.eps_p - 1e-12
    assert np.allclose(S.means(out), S.means(w), atol=1e-14)
    good = [c for c in range(S.C) if c not in bad]
    assert np.array_equal(out[good], w[good])   # tau = 1 where already positive
    assert not np.array_equal(out[bad], w[bad])


# ------------------------------------------------------------------ learned indicator (oracle)
from oracle import mlp as M


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    nin = 86
    X = rng.normal(size=(40, nin))
    y = (rng.uniform(size=40) < 0.3).astype(float)
    th = M.init_params(nin, seed=2)
    th[M.H * nin: M.H * nin + M.H] += 0.05    # nonzero biases
    loss, g = M.loss_and_grad(th, X, y)
    idx = rng.choice(len(th), 60, replace=False)
    for i in idx:
        e = np.zeros_like(th)
        e[i] = 1e-6
        num = (M.loss_and_grad(th + e, X, y)[0] - M.loss_and_grad(th - e, X, y)[0]) / 2e-6
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(g[i])


def test_mlp_features_ldf_map_is_exact():
    # the componentwise Legendre coefficients rebuild the LDF field exactly
    S = Scheme(3, 2, "powell", G, (3, 3, 3))
    w = S.project(lambda x: np.stack(np.broadcast_arrays(
        np.ones(x.shape[:-1]), 0.1 * x[..., 0], 0 * x[..., 0], 0 * x[..., 0], 2.0 + x[..., 1] ** 2,
        np.cos(3 * x[..., 1]), np.sin(2 * x[..., 2]), np.cos(x[..., 0])), -1))
    a = M.coefficients(S, w)
    u = S.eval_points(w, S.Sv)
    P = np.array([[float(v) for v in [0]] for _ in range(1)])
    from oracle import basis as OB
    Pv = np.array([OB.peval(p, S.qv) for p in S.legendre])   # [l, q]
    for c in range(3):
        rec = a[:, mhd.BX + c, :] @ Pv
        assert np.max(np.abs(rec - u[:, :, mhd.BX + c])) < 1e-12
    X = M.features(S, w)
    assert X.shape == (S.C, 86 + 24)


def test_mlp_features_octree_of_one_level_equal_uniform():
    """An octree whose leaves all have one level is the uniform mesh: the
    octree features (side averages of one leaf each, the leaf size) must equal
    the uniform ones cell by cell."""
    from oracle.amr import AMRScheme
    n = 4
    S = Scheme(3, 2, "powell", G, (n, n, n))
    leaves = [(2, (i, j, k)) for k in range(n) for j in range(n) for i in range(n)]
    A = AMRScheme(3, 2, "powell", G, leaves)
    fn = lambda x: np.stack(np.broadcast_arrays(
        1.0 + 0.3 * np.sin(2 * np.pi * x[..., 0]), 0.2 * x[..., 1], 0 * x[..., 0] + 0.1, 0 * x[..., 0],
        3.0 + np.cos(2 * np.pi * x[..., 2]), 0.5 + 0 * x[..., 0], 0.2 * np.sin(2 * np.pi * x[..., 1]),
        0 * x[..., 0] - 0.1), -1)
    wS, wA = S.project(fn), A.project(fn)
    # the same cell order (x fastest): the uniform cell index of each leaf
    idx = [(k * n + j) * n + i for (_, (i, j, k)) in leaves]
    assert np.max(np.abs(wA - wS[idx])) < 1e-13
    XS, XA = M.features(S, wS)[idx], M.features(A, wA)
    assert np.max(np.abs(XA - XS)) < 1e-12 * max(1.0, np.abs(XS).max())


def test_mlp_features_octree_side_average():
    """A coarse leaf beside four finer ones reads their average density (the
    ratio feature), a fine leaf beside a coarse one reads the coarse density,
    and the slope features scale with the leaf's own size."""
    from oracle.amr import AMRScheme
    leaves = [(1, (i, j, k)) for k in range(2) for j in range(2) for i in range(2)]
    at = leaves.index((1, (1, 0, 0)))
    kids = [(2, (2 + a, b, e)) for e in (0, 1) for b in (0, 1) for a in (0, 1)]
    leaves = leaves[:at] + kids + leaves[at + 1:]
    A = AMRScheme(3, 1, "powell", G, leaves)
    rng = np.random.default_rng(5)
    w = np.zeros((A.C, A.N))
    w[:, 0] = 1.0 + rng.uniform(0, 1, A.C)          # density means
    w[:, 4 * A.n] = 10.0                            # energy mean
    w[:, 1] = 0.01 * rng.normal(size=A.C)           # a density slope along x
    X = M.features(A, w)
    nin = 8 * A.n
    coarse = leaves.index((1, (0, 0, 0)))          # its +x side: the four kids at i = 2
    kid_rho = [w[leaves.index(kd), 0] for kd in kids if kd[1][0] == 2]
    assert len(kid_rho) == 4
    assert abs(X[coarse, nin + 1] - (np.mean(kid_rho) / w[coarse, 0] - 1.0)) < 1e-13
    fine = leaves.index((2, (2, 0, 0)))             # its -x side: the coarse leaf (0, 0, 0)
    assert abs(X[fine, nin + 0] - (w[coarse, 0] / w[fine, 0] - 1.0)) < 1e-13
    deg1x = A.modes.index((1, 0, 0))
    for c in (coarse, fine):
        assert abs(X[c, nin + 6] - w[c, deg1x] / (A.P.Mtilde * A.dxc[c])) < 1e-12


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(512, 20))
    y = (X[:, 0] + 0.5 * X[:, 3] > 0.2).astype(float)
    th = M.init_params(20, seed=1)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = M.loss_and_grad(th, X, y)[0]
    for t in range(1, 200):
        loss, g = M.loss_and_grad(th, X, y)
        th, m, v = M.adam_step(th, g, m, v, t, lr=3e-3)
    assert loss < 0.3 * l0
