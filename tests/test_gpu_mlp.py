"""Learned troubled-cell indicator on the GPU against the FP64 oracle.

* features: same definition, FP32 on the device: 2e-5 absolute
* loss and gradient (FP32 forward/backward): 1e-4 relative to the FP64 oracle
* BF16 tensor-core inference: probabilities within 0.03 of the FP64 network,
  flags equal wherever |p - 0.5| > 0.05
* training reduces the loss; gating with everything flagged equals plain TVB,
  with nothing flagged leaves the state unchanged
"""
import numpy as np
import pytest

from oracle import mhd
from oracle import mlp as M
from oracle.dg import Scheme
from oracle.limiter import Limiter

from gpu_helpers import from_device, means_to_device, rel_err, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _shock(nvar):
    def fn(x):
        r = np.sqrt((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.55) ** 2)
        inside = r < 0.27
        one = np.ones_like(r)
        u = mhd.conserved(np.where(inside, 1.0, 0.3), np.stack([0.3 * one, -0.2 * one, 0.1 * one], -1),
                          np.where(inside, 5.0, 0.2), np.stack([0.8 * one, 0.3 * one, np.where(inside, 0.2, -0.4)], -1),
                          G)
        if nvar == 9:
            u = np.concatenate([u, 0.01 * np.sin(6 * x[..., :1])], -1)
        return u
    return fn


def _slab(S):
    """Two planar discontinuities along x with smooth periodic variation in y
    and z (boxes a few cells thick in y and z)."""
    ext = np.array(S.ncell, dtype=float) * S.dx

    def fn(x):
        xs, ys, zs = x[..., 0] / ext[0], x[..., 1] / ext[1], x[..., 2] / ext[2]
        inside = (xs > 0.3) & (xs < 0.65)
        one = np.ones_like(xs)
        rho = np.where(inside, 1.0, 0.3) * (1 + 0.1 * np.sin(2 * np.pi * (ys + 2 * xs)) * np.cos(2 * np.pi * zs))
        u = mhd.conserved(rho, np.stack([0.3 * one, -0.2 * one, 0.1 * np.sin(6 * xs)], -1),
                          np.where(inside, 5.0, 0.2) * (1 + 0.2 * np.cos(2 * np.pi * (3 * xs + ys))),
                          np.stack([0.8 * one, 0.3 * one, np.where(inside, 0.2, -0.4)], -1), G)
        if S.V == 9:
            u = np.concatenate([u, 0.01 * np.sin(2 * np.pi * xs)[..., None]], -1)
        return u
    return fn


def _solver(S, prec="fp64", **kw):
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    return Solver(S.D, S.ncell, S.d, S.divb, gamma=G, box_len=S.L,
                  precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64, **kw)


@pytest.mark.parametrize("divb,prec", [("powell", "fp64"), ("glm", "fp64"), ("glm", "fp32"), ("powell", "fp32")])
def test_features(divb, prec):
    import torch
    S = Scheme(3, 2, divb, G, (7, 6, 5))
    w0 = S.project(_shock(S.V))
    sol = _solver(S, prec)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S) if prec == "fp32" else None
    X = torch.full((sol.ncell, 112), float("nan"), dtype=torch.float32, device="cuda")
    sol.mlp_features(w, wm, X, 112)
    ref = M.features(S, w0)
    got = X.cpu().numpy()
    assert ref.shape[1] == 110
    assert np.max(np.abs(got[:, :110] - ref)) < 2e-5 * max(1.0, np.abs(ref).max())
    assert np.all(got[:, 110:] == 0.0)


def test_loss_and_gradient_match_oracle():
    import torch
    from paper_1806_02343_gb300.binding import mlp_loss_grad
    rng = np.random.default_rng(3)
    n, nin = 3000, 86
    X = rng.normal(size=(n, nin))
    y = (X[:, 0] - X[:, 5] > 0.3).astype(np.uint8)
    th = M.init_params(nin, seed=4)
    th[M.H * nin:M.H * nin + M.H] = rng.normal(0, 0.1, M.H)
    loss_ref, g_ref = M.loss_and_grad(th, X, y.astype(float), pos_weight=3.0)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    thd = torch.as_tensor(th, dtype=torch.float32, device="cuda")
    loss, g = mlp_loss_grad(Xd, yd, thd, nin, pos_weight=3.0)
    assert abs(loss - loss_ref) < 1e-5 * abs(loss_ref)
    assert rel_err(g.cpu().numpy().astype(np.float64), g_ref) < 1e-4


def _train_synthetic(nin=86, n=20000, seed=0):
    import torch
    from paper_1806_02343_gb300.binding import mlp_train, mlp_loss_grad
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, nin)).astype(np.float32)
    y = (X[:, 2] + 0.5 * X[:, 7] - 0.3 * X[:, 80] > 0.8).astype(np.uint8)
    Xd = torch.as_tensor(X, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    th = torch.as_tensor(M.init_params(nin, seed=1), dtype=torch.float32, device="cuda")
    l0, _ = mlp_loss_grad(Xd, yd, th, nin)
    mlp_train(Xd, yd, th, nin, epochs=8, batch=512, lr=2e-3)
    l1, _ = mlp_loss_grad(Xd, yd, th, nin)
    return l0, l1


def test_training_reduces_loss():
    l0, l1 = _train_synthetic()
    assert l1 < 0.25 * l0


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_bf16_inference_matches_fp64_network(divb):
    import torch
    S = Scheme(3, 2, divb, G, (9, 8, 7))
    w0 = S.project(_shock(S.V))
    rng = np.random.default_rng(9)
    th = M.init_params(110, seed=5)
    th[-1] = -0.2
    sol = _solver(S)
    thd = torch.as_tensor(th, dtype=torch.float32, device="cuda")
    sol.mlp_set_weights(thd, 0.5)
    w = to_device(w0, sol)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    prob = torch.zeros(sol.stride, dtype=torch.float32, device="cuda")
    sol.mlp_infer(w, None, flags, prob)
    z, _ = M.forward(th, M.features(S, w0))
    p_ref = M.sigmoid(z)
    p = prob[: sol.ncell].cpu().numpy()
    assert np.max(np.abs(p - p_ref)) < 0.03
    sure = np.abs(p_ref - 0.5) > 0.05
    assert np.array_equal(flags[: sol.ncell].cpu().numpy()[sure].astype(bool), (p_ref > 0.5)[sure])


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_gated_tvb_limits(divb):
    import torch
    S = Scheme(3, 2, divb, G, (8, 7, 6))
    S.P.Mtilde = 0.5
    w0 = S.project(_shock(S.V))
    ref, trig = Limiter(S, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    th = M.init_params(110, seed=5)
    for b3, expect in ((40.0, ref), (-40.0, w0)):
        th[-1] = b3
        sol = _solver(S, limiter=2, Mtilde=0.5)
        if divb == "glm":
            sol.set_glm(3.0, 1.0)
        sol.mlp_set_weights(torch.as_tensor(th, dtype=torch.float32, device="cuda"), 0.5)
        w = to_device(w0, sol)
        flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
        sol.limit(w, None, flags)
        assert rel_err(from_device(w, sol), expect) < 1e-12
        f = flags[: sol.ncell].cpu().numpy().astype(bool)
        assert np.array_equal(f, trig if b3 > 0 else np.zeros_like(trig))


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_gated_tvb_partial_flags_and_counts(divb):
    """Part of the cells flagged: flagged cells get the TVB result, the others
    stay unchanged; the list-driven TVB pass counts flagged and limited cells."""
    import torch
    S = Scheme(3, 2, divb, G, (9, 7, 6))
    S.P.Mtilde = 0.5
    w0 = S.project(_shock(S.V))
    ref, trig = Limiter(S, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    th = M.init_params(110, seed=7)
    z, _ = M.forward(th, M.features(S, w0))
    th[-1] -= float(np.median(z))
    sol = _solver(S, limiter=2, Mtilde=0.5)
    if divb == "glm":
        sol.set_glm(3.0, 1.0)
    sol.mlp_set_weights(torch.as_tensor(th, dtype=torch.float32, device="cuda"), 0.5)
    w = to_device(w0, sol)
    gate = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.mlp_infer(w, None, gate, None)
    g = gate[: sol.ncell].cpu().numpy().astype(bool)
    assert 0.05 < g.mean() < 0.95
    sol.limiter_counts(reset=True)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, None, flags)
    out = from_device(w, sol)
    expect = np.where(g[:, None], ref, w0)
    assert rel_err(out, expect) < 1e-12
    f = flags[: sol.ncell].cpu().numpy().astype(bool)
    assert np.array_equal(f, trig & g)
    cnt = sol.limiter_counts()
    assert cnt == {"passes": 1, "flagged": int(g.sum()), "limited": int((trig & g).sum())}


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_staged_inference_and_gating(divb):
    """FP32 form on a mesh whose x-rows hold whole 128-cell tiles: the kernel
    that stages each tile (and its y/z neighbour tiles) in shared memory by bulk
    asynchronous copies. Probabilities within 0.03 of the FP64 network on the
    oracle's features, and the gated TVB pass equals TVB on the flagged cells."""
    import torch
    S = Scheme(3, 2, divb, G, (128, 4, 3))
    S.P.Mtilde = 0.5
    w0 = S.project(_slab(S))
    th = M.init_params(110, seed=7)
    z, _ = M.forward(th, M.features(S, w0))
    # output bias: a cut between two distinct logits near the 30th percentile
    # (uniform regions tie many cells at one logit)
    u = np.unique(z)
    k = max(1, int(np.searchsorted(u, np.sort(z)[int(0.3 * len(z))])))
    cut = 0.5 * (u[k - 1] + u[k])
    th[-1] -= cut
    p_ref = M.sigmoid(z - cut)
    sol = _solver(S, "fp32", limiter=2, Mtilde=0.5)
    if divb == "glm":
        sol.set_glm(3.0, 1.0)
    sol.mlp_set_weights(torch.as_tensor(th, dtype=torch.float32, device="cuda"), 0.5)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S)
    gate = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    prob = torch.zeros(sol.stride, dtype=torch.float32, device="cuda")
    sol.mlp_infer(w, wm, gate, prob)
    assert sol.status() == 0
    p = prob[: sol.ncell].cpu().numpy()
    assert np.max(np.abs(p - p_ref)) < 0.03
    g = gate[: sol.ncell].cpu().numpy().astype(bool)
    sure = np.abs(p_ref - 0.5) > 0.05
    assert np.array_equal(g[sure], (p_ref > 0.5)[sure])
    assert 0.05 < g.mean() < 0.95
    # gated limiting through the flagged-cell list
    ref, trig = Limiter(S, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, wm, flags)
    out = from_device(w, sol)
    expect = np.where(g[:, None], ref, w0)
    f = flags[: sol.ncell].cpu().numpy().astype(bool)
    # FP32 form against FP64 decisions: a trigger within rounding of the TVB
    # bound may flip; every other cell matches, and every flipped cell has a
    # decision quantity within FP32 rounding of its threshold
    same = f == (trig & g)
    assert same.mean() > 0.99
    assert rel_err(out[same], expect[same]) < 1e-5
    assert _flip_within_rounding(S, w0, np.nonzero(~same)[0], 3.0).all()


def _flip_within_rounding(S, w0, cells, ch, tau=1e-5):
    """For each cell whose FP32 TVB decision differs from the FP64 oracle's:
    True if FP32 rounding can decide it. The decision of a characteristic field
    (Sec. 4.2.1-4.2.2) is "|c_x| > M~ dx and |minmod(c_x, beta c+, beta c-) -
    c_x| > epsilon"; its three arguments are dot products with the left
    eigenvectors, each known to delta = tau (sum |L_kj| |slope_j| + beta sum
    |L_kj| (|D+_j| + |D-_j|)). The cell counts as within rounding if moving the
    arguments by -delta, 0 or +delta changes the decision of some field."""
    import itertools
    from oracle.limiter import eigensystem, minmod3
    Lim = Limiter(S, tvb=True, positivity=False)
    P = S.P
    m = S.means(w0)
    sl = Lim.slopes(w0)
    dpa, dma = Lim.mean_differences(m)
    thr = P.Mtilde * S.dx

    def decide(x, y, z):
        return abs(x) > thr and abs(minmod3(x, y, z) - x) > P.tvb_eps

    out = []
    for c in cells:
        near = False
        for a in range(S.D):
            R, L, _ = eigensystem(m[c], a, S.gamma, ch)
            dp, dm = dpa[c, a], dma[c, a]
            cx, cp, cm = L @ sl[c, a], L @ dp, L @ dm
            delta = tau * (np.abs(L) @ np.abs(sl[c, a]) + P.beta * (np.abs(L) @ (np.abs(dp) + np.abs(dm))))
            for k in range(S.V):
                x, y, z, dl = cx[k], P.beta * cp[k], P.beta * cm[k], delta[k]
                d0 = decide(x, y, z)
                if any(decide(x + e1 * dl, y + e2 * dl, z + e3 * dl) != d0
                       for e1, e2, e3 in itertools.product((-1, 0, 1), repeat=3)):
                    near = True
        out.append(near)
    return np.array(out, dtype=bool)


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_staged_gating_with_positivity(divb):
    """FP32 form, learned gating and positivity on the staged-kernel mesh: the
    indicator kernel screens positivity on the state it stages (unflagged cells)
    and the TVB pass lists the flagged ones. Result: positivity applied to
    (TVB on the flagged cells, the rest unchanged), with planted negative
    densities and pressures in flagged and unflagged cells."""
    import torch
    S = Scheme(3, 2, divb, G, (128, 4, 3))
    S.P.Mtilde = 0.5
    w0 = S.project(_slab(S))
    rng = np.random.default_rng(11)
    bad = rng.choice(S.C, 40, replace=False)
    w0[bad, 1] += 0.6 * np.abs(w0[bad, 0])      # rho: degree-1 mode along x
    w0[bad, 4 * S.n + 8] += 6.0 * np.abs(w0[bad, 4 * S.n])  # E: a degree-2 mode
    th = M.init_params(110, seed=7)
    z, _ = M.forward(th, M.features(S, w0))
    u = np.unique(z)
    k = max(1, int(np.searchsorted(u, np.sort(z)[int(0.3 * len(z))])))
    cut = 0.5 * (u[k - 1] + u[k])
    th[-1] -= cut
    sol = _solver(S, "fp32", limiter=2, positivity=1, Mtilde=0.5)
    if divb == "glm":
        sol.set_glm(3.0, 1.0)
    sol.mlp_set_weights(torch.as_tensor(th, dtype=torch.float32, device="cuda"), 0.5)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S)
    gate = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.mlp_infer(w, wm, gate, None)
    g = gate[: sol.ncell].cpu().numpy().astype(bool)
    assert g[bad].any() and (~g[bad]).any()
    ref_tvb, trig = Limiter(S, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    expect = Limiter(S, tvb=False, positivity=True).positivity(np.where(g[:, None], ref_tvb, w0))
    sol.counters(reset=True)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, wm, flags)
    assert sol.status() in (0, 1)
    assert sol.counters()["pos_cells"] > 0
    f = flags[: sol.ncell].cpu().numpy().astype(bool)
    same = f == (trig & g)
    assert same.mean() > 0.99
    assert _flip_within_rounding(S, w0, np.nonzero(~same)[0], 3.0).all()
    out = from_device(w, sol)
    assert rel_err(out[same], expect[same]) < 1e-5
