"""Partitioned steps on the GPU (paper_1806_02343_gb300/shard.py with the
library's SolverEngine): two ranks as threads of this process on one device
(ThreadComm: exchanges and the dt reduction on the host; no kernel waits on
another rank), each running the library on its local mesh -- a z-slab two
layers taller, or a partial octree (dg_mesh_desc.partial) -- with the
owned-cell mask for the timestep, dg_mhd_set_dt and dg_mhd_stage. One
partitioned SSP-RK3 step must equal the single-domain library step on every
owned cell: the same kernels see the same inputs, so the FP64 path agrees to
rounding of the all-reduced dt (1e-13) and the FP32 form likewise."""
import numpy as np
import pytest

from oracle.amr import AMRScheme
from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _octree():
    leaves = [(2, (i, j, k)) for k in range(4) for j in range(4) for i in range(4)]
    for c in ((1, 1, 1), (2, 1, 1), (3, 3, 0)):
        at = leaves.index((2, c))
        kids = [(3, (2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e)) for e in (0, 1) for b in (0, 1) for a in (0, 1)]
        leaves = leaves[:at] + kids + leaves[at + 1:]
    return leaves


def _blast(S):
    return S.project(lambda x: W.blast_3d(x, nvar=S.V, center=(0.3, 0.6, 0.45), r0=0.3))


CASES = [
    # (mesh, degree, scheme, precision, limited)
    (("uniform", (8, 6, 10)), 2, "glm", "fp64", True),
    (("uniform", (8, 6, 10)), 2, "glm", "fp32", True),
    (("uniform", (6, 5, 8)), 2, "powell", "fp64", True),
    (("octree", None), 1, "powell", "fp64", True),
    (("octree", None), 2, "powell", "fp32", True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0][0]}-{c[2]}-d{c[1]}-{c[3]}")
@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_step_equals_single_domain(case, world):
    import torch
    from paper_1806_02343_gb300 import binding as Bd
    from paper_1806_02343_gb300 import shard
    from gpu_helpers import means_to_device, to_device
    mesh, d, divb, prec, lim = case
    params = dict(precision=Bd.DG_PREC_FP32MIX if prec == "fp32" else Bd.DG_PREC_FP64)
    if lim:
        params.update(limiter=Bd.DG_LIMIT_TVB, positivity=1, Mtilde=0.0)
    if mesh[0] == "uniform":
        S = Scheme(3, d, divb, G, mesh[1])
        sol = Bd.Solver(3, mesh[1], d, divb, **params)
        part = shard.slab_partition(mesh[1], world)
    else:
        leaves = _octree()
        S = AMRScheme(3, d, divb, G, leaves)
        lev = np.array([l for l, _ in leaves], dtype=np.int8)
        ijk = np.array([k for _, k in leaves], dtype=np.int32)
        sol = Bd.Solver(3, None, d, divb, levels=lev, ijk=ijk, **params)
        part = shard.morton_partition(lev, ijk, world)
    w0 = _blast(S)
    # single domain
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S) if prec == "fp32" else None
    sol.step(w, wm)
    ref = w[:, : sol.ncell].double().cpu().numpy()
    refm = wm[:, : sol.ncell].cpu().numpy() if wm is not None else None
    assert sol.status() == 0

    def rank(r, comm):
        E = shard.SolverEngine(part, r, d, divb, **params)
        st = shard.ShardedSSPRK3(part, r, E, comm)
        ws, wms = E.new_state()
        lg = torch.as_tensor(part.local_global[r], device="cuda")
        full = to_device(w0, sol)
        ws[:, : len(lg)] = full[:, lg]
        if wms is not None:
            wms[:, : len(lg)] = means_to_device(w0, sol, S)[:, lg]
        st.step((ws, wms))
        torch.cuda.synchronize()
        own = np.nonzero(part.owned[r])[0]
        o = torch.as_tensor(own, device="cuda")
        return (part.local_global[r][own], ws[:, o].double().cpu().numpy(),
                None if wms is None else wms[:, o].cpu().numpy(), E.sol.status())

    res = shard.run_threads(world, rank)
    seen = np.zeros(sol.ncell, dtype=int)
    scale = np.max(np.abs(ref))
    for glob, got, gotm, status in res:
        assert status == 0
        assert np.max(np.abs(got - ref[:, glob])) <= 1e-13 * scale
        if gotm is not None:
            assert np.max(np.abs(gotm - refm[:, glob])) <= 1e-13 * np.max(np.abs(refm))
        seen[glob] += 1
    assert np.all(seen == 1)
