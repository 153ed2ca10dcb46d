"""Parity of the octree (AMR) path through the C ABI against the oracle's
AMRScheme: same-level and coarse-fine faces (Sec. 4.4). FP64 1e-12, FP32 form
on the state 1e-5."""
import numpy as np
import pytest

from oracle.amr import AMRScheme
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import from_device, means_to_device, rel_err, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _mesh(D):
    if D == 3:
        return W.octree_leaves(3, 2, 4, lambda c, dx, l: np.linalg.norm(c - 0.45) < 0.3)
    return W.octree_leaves(2, 3, 5, lambda c, dx, l: abs(c[0] - 0.5) < 0.15 or np.linalg.norm(c - 0.3) < 0.1)


def _fn(D, nvar):
    return W.SmoothFourier3D(nvar=nvar) if D == 3 else (lambda x: W.alfven_2d(x, nvar=nvar))


def _solver(A, leaves, prec="fp64", **kw):
    from paper_1806_02343_gb300.binding import Solver, DG_PREC_FP32MIX, DG_PREC_FP64
    return Solver(A.D, None, A.d, A.divb, gamma=G, box_len=1.0, leaves=leaves,
                  precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64, **kw)


@pytest.mark.parametrize("D,d,divb", [(3, 2, "powell"), (3, 2, "glm"), (2, 2, "powell"), (2, 1, "glm"), (3, 1, "powell")])
def test_amr_rhs_fp64(D, d, divb):
    leaves = _mesh(D)
    A = AMRScheme(D, d, divb, G, leaves)
    A.P.c_h_fixed = 3.0
    assert any(f[3] > 0 for f in A.faces)
    w0 = A.project(_fn(D, A.V))
    sol = _solver(A, leaves, c_h_fixed=3.0)
    if divb == "glm":
        sol.set_glm(3.0, 1.5)
    w = to_device(w0, sol)
    out = torch_nan(w)
    sol.rhs(w, None, out)
    ref = A.rhs(w0, 3.0, 1.5)
    assert rel_err(from_device(out, sol), ref) < 1e-12


@pytest.mark.parametrize("generic", [0, 1])
@pytest.mark.parametrize("d", [1, 2])
def test_amr_powell3d_both_kernel_paths(d, generic):
    """generic 0: the specialised Powell face-list kernels (faces in blocks of
    one type, B in the Legendre form of its components), 1: the generic ones;
    FP64 and the FP32 form."""
    from gpu_helpers import mean_rows
    leaves = _mesh(3)
    A = AMRScheme(3, d, "powell", G, leaves)
    assert any(f[3] == 1 for f in A.faces) and any(f[3] == 2 for f in A.faces)
    w0 = A.project(_fn(3, A.V))
    ref = A.rhs(w0, None, 0.0)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-4)):
        sol = _solver(A, leaves, prec=prec, generic_kernels=generic)
        w = to_device(w0, sol)
        out = torch_nan(w)
        if prec == "fp32":
            wm = means_to_device(w0, sol, A)
            om = torch_nan(wm)
            sol.rhs(w, wm, out, om)
            assert rel_err(om[:, : sol.ncell].cpu().numpy().T, ref[:, mean_rows(A)]) < 2e-5
        else:
            sol.rhs(w, None, out)
        assert rel_err(from_device(out, sol), ref) < tol
        assert sol.status() == 0


def torch_nan(w):
    import torch
    return torch.full_like(w, float("nan"))


@pytest.mark.parametrize("D,divb", [(3, "powell"), (2, "powell"), (3, "glm")])
def test_amr_dt_and_steps_fp64(D, divb):
    import torch
    leaves = _mesh(D)
    A = AMRScheme(D, 2, divb, G, leaves)
    A.P.c_h_fixed = 4.0
    w0 = A.project(_fn(D, A.V))
    sol = _solver(A, leaves, c_h_fixed=4.0)
    w = to_device(w0, sol)
    assert abs(sol.dt(w).item() - A.dt(w0)) <= 1e-12 * A.dt(w0)
    wo = w0.copy()
    for _ in range(2):
        sol.step(w)
        wo, _ = A.step(wo)
    assert rel_err(from_device(w, sol), wo) < 1e-11
    assert sol.status() == 0


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_amr_dt_fp32_form(divb):
    """FP32 form on an octree: an FP32 screen of every leaf, then FP64 bounds of
    the leaves within 1e-3 of the FP32 minimum, min-reduced in FP64 -- the CFL
    bound equals the oracle's to rounding; the Powell bound reads the face
    jumps of FP32 traces (5e-3, as on uniform meshes)."""
    leaves = _mesh(3)
    A = AMRScheme(3, 2, divb, G, leaves)
    A.P.c_h_fixed = 4.0
    w0 = A.project(_fn(3, A.V))
    sol = _solver(A, leaves, prec="fp32", c_h_fixed=4.0)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A)
    dt = sol.dt(w, wm).item()
    ref = A.dt(w0)
    eta = A.P.eta_powell
    A.P.eta_powell = float("inf")
    cfl_only = A.dt(w0)
    A.P.eta_powell = eta
    tol = 1e-13 if (divb == "glm" or cfl_only == ref) else 5e-3
    assert abs(dt - ref) <= tol * ref
    assert sol.status() == 0


@pytest.mark.parametrize("D,divb", [(3, "powell"), (3, "glm")])
def test_amr_fp32_form_steps(D, divb):
    import torch
    leaves = _mesh(D)
    A = AMRScheme(D, 2, divb, G, leaves)
    A.P.c_h_fixed = 4.0
    w0 = A.project(_fn(D, A.V))
    sol = _solver(A, leaves, prec="fp32", c_h_fixed=4.0)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A)
    wo = w0.copy()
    for _ in range(2):
        dto = A.dt(wo)
        sol.step(w, wm, torch.tensor([dto], dtype=torch.float64, device="cuda"))
        wo, _ = A.step(wo, dto)
    assert rel_err(from_device(w, sol), wo) < 1e-5


def _shock(nvar):
    from oracle import mhd
    def fn(x):
        r = np.sqrt(((x - 0.45) ** 2).sum(-1))
        inside = r < 0.27
        one = np.ones_like(r)
        D = x.shape[-1]
        u = mhd.conserved(np.where(inside, 1.0, 0.3), np.stack([0.3 * one, -0.2 * one, 0.1 * one], -1),
                          np.where(inside, 5.0, 0.2), np.stack([0.8 * one, 0.3 * one, np.where(inside, 0.2, -0.4)], -1),
                          G)
        if nvar == 9:
            u = np.concatenate([u, 0.01 * np.sin(6 * x[..., :1])], -1)
        return u
    return fn


@pytest.mark.parametrize("D,divb", [(3, "powell"), (3, "glm"), (2, "powell")])
def test_amr_tvb_and_positivity_fp64(D, divb):
    import torch
    from oracle.limiter import Limiter
    leaves = _mesh(D)
    A = AMRScheme(D, 2, divb, G, leaves)
    A.P.Mtilde = 0.5
    A.P.c_h_fixed = 3.0
    w0 = A.project(_shock(A.V))
    ref, trig = Limiter(A, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    sol = _solver(A, leaves, limiter=1, Mtilde=0.5, c_h_fixed=3.0)
    if divb == "glm":
        sol.set_glm(3.0, 1.0)
    w = to_device(w0, sol)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, None, flags)
    assert trig.sum() > 5
    assert np.array_equal(flags[: sol.ncell].cpu().numpy().astype(bool), trig)
    assert rel_err(from_device(w, sol), ref) < 1e-12


@pytest.mark.parametrize("divb,prec", [("powell", "fp64"), ("powell", "fp32"), ("glm", "fp64")])
def test_amr_indicator_features(divb, prec):
    """The learned indicator's features on an octree (neighbour means: the
    average of the leaves across each side; slope scale: the leaf's own size)
    against the oracle's."""
    import torch
    from oracle import mlp as M
    leaves = _mesh(3)
    A = AMRScheme(3, 2, divb, G, leaves)
    w0 = A.project(_shock(A.V))
    sol = _solver(A, leaves, prec=prec, c_h_fixed=3.0)   # (GLM on an octree takes a fixed c_h)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, A) if prec == "fp32" else None
    X = torch.full((sol.ncell, 112), float("nan"), dtype=torch.float32, device="cuda")
    sol.mlp_features(w, wm, X, 112)
    ref = M.features(A, w0)
    got = X.cpu().numpy()
    assert np.max(np.abs(got[:, :110] - ref)) < 2e-5 * max(1.0, np.abs(ref).max())
    assert np.all(got[:, 110:] == 0.0)


@pytest.mark.parametrize("divb", ["powell", "glm"])
def test_amr_gated_tvb(divb):
    """Learned indicator on an octree: part of the leaves flagged; flagged
    leaves get the octree TVB result, the others stay unchanged."""
    import torch
    from oracle import mlp as M
    from oracle.limiter import Limiter
    leaves = _mesh(3)
    A = AMRScheme(3, 2, divb, G, leaves)
    A.P.Mtilde = 0.5
    A.P.c_h_fixed = 3.0
    w0 = A.project(_shock(A.V))
    ref, trig = Limiter(A, tvb=True, positivity=False).tvb_limit(w0, 3.0)
    th = M.init_params(110, seed=7)
    z, _ = M.forward(th, M.features(A, w0))
    th[-1] -= float(np.median(z))
    sol = _solver(A, leaves, limiter=2, Mtilde=0.5, c_h_fixed=3.0)
    if divb == "glm":
        sol.set_glm(3.0, 1.0)
    sol.mlp_set_weights(torch.as_tensor(th, dtype=torch.float32, device="cuda"), 0.5)
    w = to_device(w0, sol)
    gate = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.mlp_infer(w, None, gate, None)
    g = gate[: sol.ncell].cpu().numpy().astype(bool)
    assert 0.05 < g.mean() < 0.95
    assert (trig & g).sum() > 2 and (trig & ~g).sum() > 2
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device="cuda")
    sol.limit(w, None, flags)
    assert rel_err(from_device(w, sol), np.where(g[:, None], ref, w0)) < 1e-12
    assert np.array_equal(flags[: sol.ncell].cpu().numpy().astype(bool), trig & g)
