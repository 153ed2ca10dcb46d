"""Partitioned steps (paper_1806_02343_gb300/shard.py) on CPU ranks.

The partition, the ghost lists, the exchanges (torch.distributed over gloo,
world size 2 and 3) and the stage order are the product's; each rank's
arithmetic is the FP64 oracle on that rank's local mesh (a uniform box two
layers taller, or a partial octree of the owned leaves and their face
neighbours). One partitioned SSP-RK3 step must reproduce the single-domain
oracle step on every owned cell to rounding (1e-12), with the TVB-characteristic
and positivity limiters active, and the totals must equal the single domain's.
"""
import os
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = 5.0 / 3.0


def _leaves_octree():
    """A 2:1-balanced 3D octree of 85 leaves: level 2 everywhere and three
    level-2 cells refined, two of them side by side and one at the corner of
    the periodic box (coarse-fine faces inside the box and across its wrap)."""
    from oracle.amr import balanced
    leaves = [(2, (i, j, k)) for k in range(4) for j in range(4) for i in range(4)]
    for c in ((1, 1, 1), (2, 1, 1), (3, 3, 0)):
        at = leaves.index((2, c))
        kids = [(3, (2 * c[0] + a, 2 * c[1] + b, 2 * c[2] + e)) for e in (0, 1) for b in (0, 1) for a in (0, 1)]
        leaves = leaves[:at] + kids + leaves[at + 1:]
    assert balanced(leaves, 3)
    return leaves


class OracleEngine:
    """The arithmetic of one rank with the oracle on its local mesh (test stand-in
    for the library's SolverEngine)."""

    def __init__(self, part, rank, d, divb, limiter, L=1.0):
        from oracle.amr import AMRScheme
        from oracle.dg import Scheme
        from oracle.limiter import Limiter
        kind = part.mesh[rank][0]
        P = _params(limiter)
        if kind == "uniform":
            self.S = Scheme(3, d, divb, G, part.mesh[rank][1], L=L, params=P)
            self.dxc = np.full(self.S.C, self.S.dx)
        else:
            _, lev, ijk = part.mesh[rank]
            self.S = AMRScheme(3, d, divb, G, [(int(l), tuple(int(x) for x in k)) for l, k in zip(lev, ijk)], L=L,
                               params=P)
            self.dxc = self.S.dxc
        self.own = part.owned[rank]
        self.L = Limiter(self.S, tvb=True, positivity=True) if limiter else None
        self.limits = limiter
        self.mrows = self._mean_rows()
        self.dt_val = None
        self.ch, self.kap = None, 0.0

    def _mean_rows(self):
        n = self.S.n
        if self.S.divb == "glm":
            return [v * n for v in range(9)]
        return [v * n for v in range(5)] + [5 * n + j for j in range(3)]

    def new_state(self):
        return np.zeros((self.S.C, self.S.N))

    def index(self, a):
        return np.asarray(a, dtype=np.int64)

    def pack(self, s, idx):
        return torch.from_numpy(np.ascontiguousarray(s[idx]).reshape(-1))

    def unpack(self, s, idx, buf):
        s[idx] = buf.numpy().reshape(len(idx), s.shape[1])

    def pack_means(self, s, idx):
        return torch.from_numpy(np.ascontiguousarray(s[np.ix_(idx, self.mrows)]).reshape(-1))

    def unpack_means(self, s, idx, buf):
        s[np.ix_(idx, self.mrows)] = buf.numpy().reshape(len(idx), len(self.mrows))

    def empty_like_pack(self, s, n, means_only):
        return torch.empty(n * (len(self.mrows) if means_only else s.shape[1]), dtype=torch.float64)

    def limit(self, s):
        with np.errstate(divide="ignore", invalid="ignore"):   # ghosts may miss face neighbours
            s[:] = self.L(s, self.ch)

    def dt(self, s):
        """eq. cfl and eq. powell_dt per cell (the oracle's formulas), minimum over the owned cells."""
        from oracle import mhd
        S = self.S
        m = S.means(s)
        rho, v, p, Bv = mhd.primitives(m, G)
        c = mhd.signal_speed(m, G)
        sp = np.sum(np.abs(v[:, :3]) + c[:, None], axis=1) / self.dxc
        dtc = S.P.cfl / (2 * S.d + 1) / sp
        if S.divb == "powell":
            rate = S.divb_face(s) * np.abs(np.sum(v * Bv, -1)) / m[:, mhd.EN]
            pos = rate > 0
            dtc = np.where(pos, np.minimum(dtc, S.P.eta_powell / np.where(pos, rate, 1.0)), dtc)
        return torch.tensor([np.min(dtc[self.own])], dtype=torch.float64)

    def set_dt(self, t):
        self.dt_val = float(t[0])
        if self.S.divb == "glm":
            self.ch, self.kap = self.S.glm_speeds(self.dt_val)

    def stage(self, w, u0, out, a, b):
        r = self.S.rhs(w, self.ch, self.kap)
        res = b * (w + self.dt_val * r)
        if u0 is not None:
            res = a * u0 + res
        out[:] = res

    def totals(self, s):
        t = (self.S.means(s) * (self.dxc ** 3)[:, None])[self.own].sum(0)
        return torch.from_numpy(np.ascontiguousarray(t))


def _params(limited):
    """M~ = 0 with the limiters (pure minmod, Sec. 4.2.1): on these coarse meshes
    the default M~ dx exceeds every slope, and detection would never compare a
    cell with its neighbours' means."""
    from oracle.dg import Params
    return Params(Mtilde=0.0) if limited else Params()


def _state(S, divb, kind):
    from paper_1806_02343_gb300 import workloads as W
    if kind == "blast":
        return S.project(lambda x: W.blast_3d(x, nvar=S.V, center=(0.3, 0.6, 0.45), r0=0.3))
    return S.project(W.SmoothFourier3D(nvar=S.V))


def _single(case):
    """Single-domain oracle: mesh, start, one step (with limiters if asked)."""
    from oracle.amr import AMRScheme
    from oracle.dg import Scheme
    from oracle.limiter import Limiter
    mesh, d, divb, lim, kind = case
    P = _params(lim)
    S = Scheme(3, d, divb, G, mesh[1], params=P) if mesh[0] == "uniform" else AMRScheme(3, d, divb, G, mesh[1],
                                                                                       params=P)
    w0 = _state(S, divb, kind)
    Lm = Limiter(S, tvb=True, positivity=True) if lim else None
    if Lm is not None:
        with np.errstate(divide="ignore", invalid="ignore"):
            w1, dt = S.step(w0, limiter=lambda x: Lm(x, None))
    else:
        w1, dt = S.step(w0)
    return S, w0, w1, dt


def _partition(case, world):
    from paper_1806_02343_gb300 import shard
    mesh = case[0]
    if mesh[0] == "uniform":
        return shard.slab_partition(mesh[1], world)
    lev = np.array([l for l, _ in mesh[1]], dtype=np.int8)
    ijk = np.array([k for _, k in mesh[1]], dtype=np.int32)
    return shard.morton_partition(lev, ijk, world)


def _run_rank(rank, world, case, part, w0, comm):
    from paper_1806_02343_gb300 import shard
    mesh, d, divb, lim, kind = case
    E = OracleEngine(part, rank, d, divb, lim)
    st = shard.ShardedSSPRK3(part, rank, E, comm)
    s = np.ascontiguousarray(w0[part.local_global[rank]])
    tot0 = st.totals(s).numpy().copy()
    dt = float(st.step(s)[0])
    own = part.owned[rank]
    return part.local_global[rank][own], s[own], dt, tot0


def _rank_main(rank, world, port, case, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1806_02343_gb300 import shard
    S, w0, _, _ = _single(case)
    part = _partition(case, world)
    out[rank] = _run_rank(rank, world, case, part, w0, shard.TorchComm(rank, world))
    dist.barrier()
    dist.destroy_process_group()


UNIFORM = ("uniform", (4, 3, 6))


def _octree_case():
    return ("octree", _leaves_octree())


CASES = {
    "uniform_glm": (UNIFORM, 1, "glm", False, "smooth"),
    "uniform_powell_limited": (UNIFORM, 2, "powell", True, "blast"),
    "octree_powell_limited": (None, 1, "powell", True, "blast"),
}


def _case(name):
    c = CASES[name]
    if c[0] is None:
        c = (_octree_case(),) + c[1:]
    return c


def _check(case, results):
    S, w0, w1, dt = _single(case)
    seen = np.zeros(S.C, dtype=int)
    scale = np.max(np.abs(w1))
    for glob, loc, dtr, tot0 in results:
        assert abs(dtr - dt) <= 1e-13 * dt
        assert np.max(np.abs(loc - w1[glob])) <= 1e-12 * scale
        assert np.allclose(tot0, S.totals(w0), rtol=1e-13, atol=1e-15)
        seen[glob] += 1
    assert np.all(seen == 1)


@pytest.mark.parametrize("name", list(CASES))
def test_partition_lists_are_consistent(name):
    """Every cell owned once; the ghost lists pair up across ranks; every face
    neighbour of an owned cell (from the oracle's own face list) is local."""
    case = _case(name)
    S, _, _, _ = _single(case)
    for world in (1, 2, 3):
        part = _partition(case, world)
        owned = np.concatenate([part.local_global[r][part.owned[r]] for r in range(world)])
        assert np.array_equal(np.sort(owned), np.arange(S.C))
        for r in range(world):
            for q in range(world):
                a = part.local_global[q][part.sends[q][r]]
                b = part.local_global[r][part.recvs[r][q]]
                assert np.array_equal(a, b)
                assert np.all(part.owned[q][part.sends[q][r]]) and not np.any(part.owned[r][part.recvs[r][q]])
        nb = [set() for _ in range(S.C)]
        if case[0][0] == "uniform":
            for a in range(3):
                for c in range(S.C):
                    nb[c].add(int(S.nbr_plus[a][c]))
                    nb[c].add(int(S.nbr_minus[a][c]))
        else:
            for cL, cR, *_ in S.faces:
                nb[cL].add(cR)
                nb[cR].add(cL)
        for r in range(world):
            local = set(part.local_global[r].tolist())
            for g in part.local_global[r][part.owned[r]]:
                assert nb[g] <= local


@pytest.mark.parametrize("name", list(CASES))
def test_one_rank_with_periodic_ghosts_matches_single_domain(name):
    """World size 1: the ghosts are the rank's own cells across the wrap (uniform)
    or none (octree); no process group is needed."""
    from paper_1806_02343_gb300 import shard
    case = _case(name)
    S, w0, _, _ = _single(case)
    part = _partition(case, 1)
    _check(case, [_run_rank(0, 1, case, part, w0, shard.TorchComm(0, 1))])


@pytest.mark.parametrize("name,world", [("uniform_glm", 2), ("uniform_powell_limited", 2),
                                        ("octree_powell_limited", 2), ("octree_powell_limited", 3)])
def test_gloo_ranks_match_single_domain(name, world):
    case = _case(name)
    port = 29600 + (os.getpid() % 1500) + 7 * world
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, case, out), nprocs=world, join=True)
        res = [out[r] for r in range(world)]
    _check(case, res)


@pytest.mark.parametrize("name", ["uniform_powell_limited", "octree_powell_limited"])
def test_thread_ranks_match_single_domain(name):
    """The same partitioned step with the ranks as threads of one process
    (ThreadComm: host-side queues and a barrier)."""
    from paper_1806_02343_gb300 import shard
    case = _case(name)
    S, w0, _, _ = _single(case)
    part = _partition(case, 2)
    res = shard.run_threads(2, lambda r, comm: _run_rank(r, 2, case, part, w0, comm))
    _check(case, res)
