"""Partitioned DG-MHD steps across ranks (one process per GPU).

The operator of Sec. 3.5 (eq. wdot) couples a cell only to its face
neighbours -- the compact stencil the paper credits DG with (Sec. 1 and the
discussion of Sec. 6) -- so the mesh shards into contiguous ranges of cells:
z-slabs of a uniform box, or contiguous ranges of the Morton order of an
octree's leaves. Each rank keeps its owned cells plus one layer of ghost cells,
the face neighbours of its owned cells that another rank owns, and runs the
unchanged single-mesh library on that local mesh (a uniform box two layers
taller, or a partial octree). Ghost results are never used; per RK stage two
exchanges refresh the ghosts:

1. the cell means before the limiter (the TVB detection compares a cell's
   slopes with its neighbours' means, Sec. 4.2.1);
2. the whole limited state after it (the face fluxes read the traces of both
   neighbours, Sec. 4.1.2);

and per step one MIN all-reduce of the CFL step (eq. cfl, eq. powell_dt) over
the owned cells. `totals` adds one SUM all-reduce of the FP64 conservation
totals. Remote data lands in local buffers first (point-to-point send/recv into
staging tensors); no kernel reads a peer's memory.

The arithmetic per rank is the library's (through an engine object: the
binding's Solver for the GPU); this module holds the partition, the exchange
lists, the communication and the stage order of the SSP-RK3 step of Sec. 3.6
(limiter before every stage evaluation, Sec. 4.3), and nothing of the method's
arithmetic.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------- partitions


class Partition:
    """Cell ownership and ghost lists of a partitioned mesh.

    local_global[r]   global cell index of each cell of rank r's local mesh
    owned[r]          bool per local cell: rank r owns it
    sends[r][q]       local indices (in r's numbering) of r's owned cells that
                      rank q holds as ghosts, in increasing global index
    recvs[r][q]       local indices (in r's numbering) of r's ghosts owned by
                      q, in increasing global index (so recvs[r][q] matches
                      sends[q][r] element by element)
    mesh[r]           the local mesh: ("uniform", (nx, ny, nz)) or
                      ("octree", levels, ijk) of a partial octree
    """

    def __init__(self, world, local_global, owned, owner_of_global, mesh):
        self.world = world
        self.local_global = [np.asarray(x, dtype=np.int64) for x in local_global]
        self.owned = [np.asarray(x, dtype=bool) for x in owned]
        self.mesh = mesh
        # where each global cell's owned instance sits in its owner's local mesh
        owned_local = {}
        for r in range(world):
            idx = np.nonzero(self.owned[r])[0]
            owned_local[r] = (self.local_global[r][idx], idx)
        self.sends = [[np.zeros(0, dtype=np.int64) for _ in range(world)] for _ in range(world)]
        self.recvs = [[np.zeros(0, dtype=np.int64) for _ in range(world)] for _ in range(world)]
        for r in range(world):
            ghost = np.nonzero(~self.owned[r])[0]
            g_glob = self.local_global[r][ghost]
            g_own = owner_of_global(g_glob)
            for q in range(world):
                sel = g_own == q
                if not np.any(sel):
                    continue
                order = np.argsort(g_glob[sel], kind="stable")
                gl = g_glob[sel][order]
                self.recvs[r][q] = ghost[sel][order]
                og, oi = owned_local[q]
                srt = np.argsort(og, kind="stable")
                pos = np.searchsorted(og[srt], gl)
                if np.any(pos >= len(og)) or np.any(og[srt][np.minimum(pos, len(og) - 1)] != gl):
                    raise ValueError("a ghost cell's owner does not hold it")
                self.sends[q][r] = oi[srt][pos]

    def n_local(self, r):
        return len(self.local_global[r])


def slab_partition(n, world):
    """z-slabs of a uniform periodic box of n = (nx, ny, nz) cells (x fastest):
    rank r owns the layers [z0_r, z0_{r+1}) (contiguous cell ranges, the
    Morton-free special case of a contiguous partition) and holds one ghost
    layer below and one above; its local mesh is a uniform box of nz_r + 2
    layers (periodic in z too, which only couples the two ghost layers, whose
    results are discarded)."""
    nx, ny, nz = (int(x) for x in n)
    if world < 1 or nz < world:
        raise ValueError("need at least one z-layer per rank")
    bounds = [(r * nz) // world for r in range(world + 1)]
    A = nx * ny
    local_global, owned, mesh = [], [], []
    for r in range(world):
        z0, z1 = bounds[r], bounds[r + 1]
        nl = z1 - z0
        zl = np.arange(nl + 2)
        gz = (z0 - 1 + zl) % nz
        lg = (gz[:, None] * A + np.arange(A)[None, :]).reshape(-1)
        own = np.zeros((nl + 2, A), dtype=bool)
        own[1:nl + 1] = True
        local_global.append(lg)
        owned.append(own.reshape(-1))
        mesh.append(("uniform", (nx, ny, nl + 2)))
    owner_z = np.zeros(nz, dtype=np.int64)
    for r in range(world):
        owner_z[bounds[r]:bounds[r + 1]] = r

    def owner_of(g):
        return owner_z[np.asarray(g) // A]

    return Partition(world, local_global, owned, owner_of, mesh)


def morton_codes(levels, ijk):
    """Morton (Z-order) codes of octree leaves at the finest level present:
    the bits of the coordinates interleaved, x lowest."""
    lev = np.asarray(levels, dtype=np.int64)
    k = np.asarray(ijk, dtype=np.int64).reshape(len(lev), -1)
    D = k.shape[1]
    R = int(lev.max()) if len(lev) else 0
    scaled = k << (R - lev)[:, None]
    code = np.zeros(len(lev), dtype=np.uint64)
    for b in range(R + 1):
        for a in range(D):
            bit = ((scaled[:, a] >> b) & 1).astype(np.uint64)
            code |= bit << np.uint64(D * b + a)
    return code


def morton_partition(levels, ijk, world, faces=None):
    """Contiguous ranges of the Morton order of an octree's leaves, balanced by
    count. Ghosts: the cells across every face (same-level and coarse-fine)
    from one rank's cell to another's. `faces` = (left, right) arrays of the
    face list; by default the library's own (binding.octree_faces). Each local
    mesh lists its cells in increasing global index (the input order)."""
    lev = np.asarray(levels, dtype=np.int8)
    k = np.asarray(ijk, dtype=np.int32).reshape(len(lev), -1)
    N = len(lev)
    if world < 1 or N < world:
        raise ValueError("need at least one leaf per rank")
    order = np.argsort(morton_codes(lev, k), kind="stable")
    owner = np.zeros(N, dtype=np.int64)
    bounds = [(r * N) // world for r in range(world + 1)]
    for r in range(world):
        owner[order[bounds[r]:bounds[r + 1]]] = r
    if faces is None:
        from . import binding
        fl, fr, _ = binding.octree_faces(lev, k)
    else:
        fl, fr = faces
    fl = np.asarray(fl, dtype=np.int64)
    fr = np.asarray(fr, dtype=np.int64)
    cross = owner[fl] != owner[fr]
    local_global, owned, mesh = [], [], []
    for r in range(world):
        mine = owner == r
        ghosts = np.concatenate([fl[cross & (owner[fr] == r)], fr[cross & (owner[fl] == r)]])
        cells = np.union1d(np.nonzero(mine)[0], ghosts)
        local_global.append(cells)
        owned.append(owner[cells] == r)
        mesh.append(("octree", lev[cells].copy(), k[cells].copy()))
    return Partition(world, local_global, owned, lambda g: owner[np.asarray(g)], mesh)


# --------------------------------------------------------------- communication


class TorchComm:
    """Point-to-point exchange and reductions over torch.distributed (NCCL
    between GPUs, gloo on CPU); world size 1 needs no process group."""

    def __init__(self, rank, world, group=None):
        self.rank, self.world, self.group = rank, world, group

    def exchange(self, send, recv_like):
        """send[q]: tensor for rank q (or None); recv_like[q]: empty tensor to
        fill from rank q (or None). Self-sends are copies."""
        import torch.distributed as dist
        out = {}
        ops = []
        for q in range(self.world):
            if q == self.rank:
                if send[q] is not None:
                    out[q] = send[q].clone()
                continue
            if recv_like[q] is not None:
                out[q] = recv_like[q]
                ops.append(dist.P2POp(dist.irecv, out[q], q, self.group))
            if send[q] is not None:
                ops.append(dist.P2POp(dist.isend, send[q], q, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return out

    def allreduce_min(self, t):
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return t

    def allreduce_sum(self, t):
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t


class ThreadComm:
    """The ranks as threads of one process (several devices driven from one
    host process, or a partition checked on one device): exchanges go through
    host-side queues, reductions through a barrier. No kernel waits on another
    rank; every wait is on the host and bounded by `timeout_s`."""

    class Hub:
        def __init__(self, world, timeout_s=120.0):
            import queue
            import threading
            self.world, self.timeout = world, timeout_s
            self.q = {(a, b): queue.Queue() for a in range(world) for b in range(world)}
            self.bar = threading.Barrier(world, timeout=timeout_s)
            self.slots = [None] * world

    def __init__(self, rank, hub):
        self.rank, self.world, self.hub = rank, hub.world, hub

    def exchange(self, send, recv_like):
        for q in range(self.world):
            if send[q] is not None:
                self.hub.q[(self.rank, q)].put(send[q].clone() if q == self.rank else send[q])
        out = {}
        for q in range(self.world):
            if recv_like[q] is not None:
                out[q] = self.hub.q[(q, self.rank)].get(timeout=self.hub.timeout)
        return out

    def _reduce(self, t, op):
        self.hub.slots[self.rank] = t
        self.hub.bar.wait()
        acc = self.hub.slots[0].clone()
        for x in self.hub.slots[1:]:
            acc = op(acc, x.to(acc.device))
        self.hub.bar.wait()
        t.copy_(acc)
        return t

    def allreduce_min(self, t):
        import torch
        return self._reduce(t, torch.minimum)

    def allreduce_sum(self, t):
        return self._reduce(t, lambda a, b: a + b)


def run_threads(world, fn, timeout_s=600.0):
    """fn(rank, comm) on `world` threads sharing a ThreadComm hub; returns the
    per-rank results (re-raises the first exception)."""
    import threading
    hub = ThreadComm.Hub(world)
    res, err = [None] * world, []

    def body(r):
        try:
            res[r] = fn(r, ThreadComm(r, hub))
        except BaseException as e:  # surfaced to the caller below
            err.append(e)
            hub.bar.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout_s)
    if err:
        raise err[0]
    if any(t.is_alive() for t in th):
        raise TimeoutError("a rank thread did not finish")
    return res


# ------------------------------------------------------------------ stepping


class ShardedSSPRK3:
    """One rank's SSP-RK3 step (Sec. 3.6, Shu-Osher form) on a partitioned
    mesh, in the stage order of dg_mhd_step: limit u^n, dt from the limited
    state (MIN over the ranks), then three stages, the second and third
    inputs limited first; ghosts refreshed before every limiter pass (means)
    and after it (whole state).

    engine: the rank's arithmetic with the methods
        new_state(), limit(s), dt(s) -> 1-element float64 tensor (owned cells),
        set_dt(t), stage(w, u0, out, a, b) (out = a u0 + b (w + dt L(w))),
        pack(s, idx), unpack(s, idx, buf), pack_means(s, idx),
        unpack_means(s, idx, buf), totals(s) -> float64 tensor (owned cells),
        and the flag `limits` (a limiter pass runs).
    """

    def __init__(self, part, rank, engine, comm):
        self.part, self.rank, self.E, self.comm = part, rank, engine, comm
        self.s1 = engine.new_state()
        self.s2 = engine.new_state()
        self._idx = {}

    def _t(self, a):
        key = id(a)
        if key not in self._idx:
            self._idx[key] = self.E.index(a)
        return self._idx[key]

    def exchange(self, s, means_only=False):
        p, r = self.part, self.rank
        pack = self.E.pack_means if means_only else self.E.pack
        unpack = self.E.unpack_means if means_only else self.E.unpack
        send, like = {}, {}
        for q in range(p.world):
            si, ri = p.sends[r][q], p.recvs[r][q]
            send[q] = pack(s, self._t(si)) if len(si) else None
            like[q] = self.E.empty_like_pack(s, len(ri), means_only) if len(ri) else None
        got = self.comm.exchange(send, like)
        for q, buf in got.items():
            unpack(s, self._t(p.recvs[r][q]), buf)

    def limit(self, s):
        if self.E.limits:
            self.exchange(s, means_only=True)
            self.E.limit(s)
        self.exchange(s)

    def step(self, s):
        """Advances s in place by one step; returns the step length (tensor)."""
        E = self.E
        self.limit(s)
        dt = self.comm.allreduce_min(E.dt(s))
        E.set_dt(dt)
        E.stage(s, None, self.s1, 0.0, 1.0)
        self.limit(self.s1)
        E.stage(self.s1, s, self.s2, 0.75, 0.25)
        self.limit(self.s2)
        E.stage(self.s2, s, s, 1.0 / 3.0, 2.0 / 3.0)
        return dt

    def totals(self, s):
        """Volume integrals of the conserved variables over the whole mesh (FP64,
        SUM over the ranks of the owned cells' sums)."""
        return self.comm.allreduce_sum(self.E.totals(s))


class SolverEngine:
    """The library's Solver on a rank's local mesh (GPU): the arithmetic of
    ShardedSSPRK3. Local meshes come from Partition.mesh (a uniform box, or a
    partial octree); the owned-cell mask restricts the timestep minimum."""

    def __init__(self, part, rank, degree, divb, box_len=1.0, device="cuda", **params):
        import torch
        from .binding import Solver
        kind = part.mesh[rank][0]
        if kind == "uniform":
            nloc = part.mesh[rank][1]
            dx = box_len / nloc[0]
            self.sol = Solver(3, nloc, degree, divb, box_len=dx * nloc[0], **params)
        else:
            _, lev, ijk = part.mesh[rank]
            self.sol = Solver(ijk.shape[1], None, degree, divb, box_len=box_len, levels=lev, ijk=ijk, partial=True,
                              **params)
        self.device = torch.device(device)
        own = torch.as_tensor(part.owned[rank].astype(np.uint8), device=self.device)
        self.owned = own.bool()
        self.sol.set_owned(own)
        self.limits = self.sol.params.limiter != 0 or self.sol.params.positivity != 0
        self.fp32 = self.sol.fp32
        self.mrows = self.sol.mean_rows()
        self._dt = torch.zeros(1, dtype=torch.float64, device=self.device)
        self._vol = None

    def new_state(self):
        return self.sol.alloc_state(self.device)

    def index(self, a):
        import torch
        return torch.as_tensor(np.asarray(a, dtype=np.int64), device=self.device)

    def pack(self, s, idx):
        # the FP64 means first, so that every view of the byte buffer is aligned
        import torch
        w, wm = s
        parts = [w[:, idx].contiguous().view(-1).view(torch.uint8)]
        if wm is not None:
            parts.insert(0, wm[:, idx].contiguous().view(-1).view(torch.uint8))
        return torch.cat(parts)

    def unpack(self, s, idx, buf):
        import torch
        w, wm = s
        nm = wm.shape[0] * len(idx) * 8 if wm is not None else 0
        if wm is not None:
            wm[:, idx] = buf[:nm].view(torch.float64).view(wm.shape[0], len(idx))
        w[:, idx] = buf[nm:].view(w.dtype).view(w.shape[0], len(idx))

    def pack_means(self, s, idx):
        import torch
        w, wm = s
        m = wm[:, idx] if wm is not None else w[self.mrows][:, idx]
        return m.contiguous().view(-1).view(torch.uint8)

    def unpack_means(self, s, idx, buf):
        import torch
        w, wm = s
        if wm is not None:
            m = buf.view(torch.float64).view(wm.shape[0], len(idx))
            wm[:, idx] = m
            # the float mirror rows of the FP32 form follow their FP64 means
            w[torch.as_tensor(self.mrows, device=w.device)[:, None], idx[None, :]] = m.to(w.dtype)
        else:
            m = buf.view(w.dtype).view(len(self.mrows), len(idx))
            w[torch.as_tensor(self.mrows, device=w.device)[:, None], idx[None, :]] = m

    def empty_like_pack(self, s, n, means_only):
        import torch
        w, wm = s
        if means_only:
            nbytes = (wm.shape[0] * 8 if wm is not None else len(self.mrows) * w.element_size()) * n
        else:
            nbytes = w.shape[0] * w.element_size() * n + (wm.shape[0] * 8 * n if wm is not None else 0)
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def limit(self, s):
        self.sol.limit(s[0], s[1])

    def dt(self, s):
        return self.sol.dt(s[0], s[1], out=self._dt)

    def set_dt(self, t):
        self.sol.set_dt(t)

    def stage(self, w, u0, out, a, b):
        self.sol.stage(w[0], w[1], None if u0 is None else u0[0], None if u0 is None else u0[1], out[0], out[1],
                       a, b)

    def totals(self, s):
        import torch
        w, wm = s
        n = self.sol.ncell
        m = (wm[:, :n] if wm is not None else w[self.mrows, :n]).to(torch.float64)
        if self._vol is None:
            if self.sol._lev is not None:
                dx = self.sol.box_len / (2.0 ** torch.as_tensor(self.sol._lev.astype(np.float64), device=w.device))
                self._vol = dx ** self.sol.dim
            else:
                dx = self.sol.box_len / self.sol._n[0]
                self._vol = torch.full((n,), dx ** self.sol.dim, dtype=torch.float64, device=w.device)
        return (m * (self._vol * self.owned[:n])[None, :]).sum(1)
