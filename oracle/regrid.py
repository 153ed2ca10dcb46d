"""Oracle of dynamic octree regridding (test infrastructure only: only the
tests, the smoke check and the benchmark's CPU legs import it; the CUDA path
never does). It follows Sec. 5 (adaptive mesh refinement) of the paper:

* prolongation: the weights of child o are the L2 projection of the parent's
  polynomial, restricted to octant o, onto the child's basis -- per variable
  for the Legendre rows, under the vector inner product of eq. innerp for the
  LDF rows (a divergence-free parent field is represented exactly);
* restriction: the L2 projection onto the parent's basis of the field formed by
  the 2^D children;
* smoothness indicator S_a(u) = sum_{k=1..d} 2^(2k-1) int (d^k u / dxi_a^k)^2
  over the reference cell, for each monitored conserved component u (the B
  components of the Powell form evaluated from its LDF rows);
* marks: a leaf is refined if S_a(u) > 2 S~ for any monitored u and direction
  a; a split cell -- here a group of 2^D sibling leaves -- is coarsened if the
  restriction of its children has S_a(u) < S~ / 2 for every monitored u and
  direction;
* the new leaf list (readings, the paper defers the details to its refs):
  refinement below max_level only, coarsening above min_level only and never
  of a group with a member marked for refinement; then 2:1 balance across
  faces, first by refining every leaf that is two levels coarser than a face
  neighbour (repeated until none is), then by cancelling every coarsening whose
  parent would be two levels coarser than a neighbour (repeated as well).

Octant o of a parent: bit a of o set = upper half along axis a; child
coordinates k_a = 2 k_a(parent) + bit a; the child's reference point xi maps
to the parent's (xi + s) / 2 with s_a = +1 (bit set) or -1.

Exact rationals (oracle.basis polynomials) build the matrices; the smoothness
indicator uses the Gauss rule with d+1 points per dimension, exact for the
squared derivatives (degree <= 2d - 2).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb

import numpy as np

from . import basis as B
from . import mhd


# ----------------------------------------------------------------- polynomials
def affine_octant(poly: dict, s: tuple) -> dict:
    """poly((xi + s) / 2) as a polynomial in xi (s_a = +1 or -1 per axis)."""
    out: dict = {}
    for e, c in poly.items():
        # prod_a ((x_a + s_a) / 2)^e_a = prod_a sum_j C(e_a, j) x_a^j s_a^(e_a-j) / 2^e_a
        terms = {tuple([0] * len(e)): c}
        for a, ea in enumerate(e):
            nxt: dict = {}
            for te, tc in terms.items():
                for j in range(ea + 1):
                    ne = list(te)
                    ne[a] += j
                    v = tc * comb(ea, j) * Fraction(s[a]) ** (ea - j) / Fraction(2) ** ea
                    if v != 0:
                        nxt[tuple(ne)] = nxt.get(tuple(ne), 0) + v
            terms = nxt
        for te, tc in terms.items():
            v = out.get(te, 0) + tc
            if v == 0:
                out.pop(te, None)
            else:
                out[te] = v
    return out


def octant_sign(o: int, D: int) -> tuple:
    return tuple(1 if (o >> a) & 1 else -1 for a in range(D))


# ------------------------------------------------------------ row polynomials
def _row_fields(S):
    """Per row r: (kind, var, polys) with polys the D components (LDF) or the
    scalar Legendre polynomial of the row."""
    out = []
    for kind, v, i in S.rows:
        if kind == "L":
            out.append(("L", v, S.legendre[i]))
        else:
            out.append(("B", None, S.ldf[i]))
    return out


@lru_cache(maxsize=None)
def _prolongation_exact(D: int, d: int, divb: str) -> tuple:
    """Exact prolongation matrices Pr[o][r_child][r_parent] (Fractions) for the
    row layout of oracle.dg.Scheme(D, d, divb)."""
    from .dg import Scheme
    S = Scheme(D, d, divb, 5.0 / 3.0, 2)
    rows = _row_fields(S)
    N = len(rows)
    mats = []
    for o in range(2 ** D):
        s = octant_sign(o, D)
        P = [[Fraction(0)] * N for _ in range(N)]
        for rp, (kp, vp, pp) in enumerate(rows):
            if kp == "L":
                shifted = affine_octant(pp, s)
                for rc, (kc, vc, pc) in enumerate(rows):
                    if kc == "L" and vc == vp:
                        P[rc][rp] = B.pintegrate(B.pmul(shifted, pc)) / S.mass_exact[rc]
            else:
                shifted = tuple(affine_octant(c, s) if c else {} for c in pp)
                for rc, (kc, vc, pc) in enumerate(rows):
                    if kc == "B":
                        P[rc][rp] = B.vdot(shifted, pc) / S.mass_exact[rc]
        mats.append(P)
    return tuple(tuple(tuple(r) for r in P) for P in mats), tuple(S.mass_exact)


def prolongation(S) -> np.ndarray:
    """Pr[o, r_child, r_parent] in float64 for the scheme S's row layout."""
    P, _ = _prolongation_exact(S.D, S.d, S.divb)
    return np.array([[[float(x) for x in row] for row in Po] for Po in P])


def restriction(S) -> np.ndarray:
    """Re[o, r_parent, r_child]: the parent's weights are sum_o Re[o] @ w_child[o].
    From the change of variables xi_parent = (xi_child + s) / 2 (volume ratio
    2^-D) the projection onto the parent's row r of child o's row r' is
    2^-D M_r' / M_r times the prolongation entry Pr[o, r', r]."""
    P, mass = _prolongation_exact(S.D, S.d, S.divb)
    N = len(mass)
    out = np.zeros((2 ** S.D, N, N))
    for o in range(2 ** S.D):
        for r in range(N):
            for rc in range(N):
                if P[o][rc][r] != 0:
                    out[o, r, rc] = float(P[o][rc][r] * mass[rc] / mass[r] / 2 ** S.D)
    return out


def prolong(S, w_parent: np.ndarray) -> np.ndarray:
    """Children weights [2^D, N] of one parent's weights [N]."""
    return np.einsum("oab,b->oa", prolongation(S), w_parent)


def restrict(S, w_children: np.ndarray) -> np.ndarray:
    """Parent weights [N] of the 2^D children's weights [2^D, N]."""
    return np.einsum("oab,ob->a", restriction(S), w_children)


# ------------------------------------------------------- smoothness indicator
@lru_cache(maxsize=None)
def _deriv_tables(D: int, d: int, divb: str):
    """T[k-1][a][r, q, v]: k-th derivative along axis a of row r's component v
    at the Gauss points (d+1 per dimension), k = 1..d; and the weights."""
    from .dg import Scheme
    S = Scheme(D, d, divb, 5.0 / 3.0, 2)
    pts, wts = B.gauss_tensor(D, d + 1)
    T = np.zeros((d, D, S.N, len(wts), S.V))
    for r, (kind, v, i) in enumerate(S.rows):
        comps = [(v, S.legendre[i])] if kind == "L" else [(mhd.BX + a, c) for a, c in enumerate(S.ldf[i]) if c]
        for a in range(D):
            for vv, poly in comps:
                p = poly
                for k in range(1, d + 1):
                    p = B.pderiv(p, a)
                    if p:
                        T[k - 1, a, r, :, vv] = B.peval(p, pts)
    return T, wts


def smoothness(S, w: np.ndarray, fields) -> np.ndarray:
    """S_a(u) for the rows w[C, N] of C cells: array [C, len(fields), D] for the
    monitored conserved components `fields` (indices into the V variables)."""
    T, wts = _deriv_tables(S.D, S.d, S.divb)
    w = np.atleast_2d(w)
    out = np.zeros((w.shape[0], len(fields), S.D))
    for k in range(1, S.d + 1):
        for a in range(S.D):
            vals = np.einsum("cr,rqv->cqv", w, T[k - 1, a])  # d^k u / dxi_a^k at the points
            for j, f in enumerate(fields):
                out[:, j, a] += 2.0 ** (2 * k - 1) * np.einsum("cq,q->c", vals[:, :, f] ** 2, wts)
    return out


# ------------------------------------------------------------------- the mesh
def sibling_groups(leaves, D):
    """Groups of 2^D leaves that are the children of one parent, sorted by
    (parent level, parent coordinates): list of (parent_level, parent_ijk,
    [leaf index of octant o for o = 0 .. 2^D - 1])."""
    idx = {(l,) + tuple(k): c for c, (l, k) in enumerate(leaves)}
    groups = {}
    for l, k in leaves:
        if l == 0:
            continue
        pk = tuple(x // 2 for x in k)
        if (l - 1, pk) in groups:
            continue
        mem = [idx.get((l,) + tuple(2 * pk[a] + ((o >> a) & 1) for a in range(D))) for o in range(2 ** D)]
        groups[(l - 1, pk)] = mem if all(m is not None for m in mem) else None
    return [(pl, pk, mem) for (pl, pk), mem in sorted(groups.items()) if mem is not None]


def marks(S, leaves, w, fields, Stilde, min_level, max_level):
    """Refinement marks of Sec. 5: refine[C] (leaves with S_a(u) > 2 S~ for some
    monitored u and direction a, below max_level) and the indices of the sibling
    groups to coarsen (restriction with S_a(u) < S~/2 for all, parent level >=
    min_level, no member marked for refinement)."""
    sm = smoothness(S, w, fields).reshape(len(leaves), -1).max(axis=1)
    refine = np.array([sm[c] > 2.0 * Stilde and l < max_level for c, (l, _) in enumerate(leaves)], dtype=bool)
    groups = sibling_groups(leaves, S.D)
    coarsen = []
    for g, (pl, _, mem) in enumerate(groups):
        if pl < min_level or refine[mem].any():
            continue
        wp = restrict(S, w[mem])
        if smoothness(S, wp[None], fields).max() < 0.5 * Stilde:
            coarsen.append(g)
    return refine, groups, coarsen


def _covering_level(mesh, l, k):
    """Level of the leaf of `mesh` that contains the cube (l, k), None if the
    cube is split into finer leaves."""
    for ll in range(l, -1, -1):
        if (ll, tuple(x >> (l - ll) for x in k)) in mesh:
            return ll
    return None


def _face_ok(mesh, l, k, D):
    """No face neighbour of the cube (l, k) holds leaves of level >= l + 2."""
    n = 2 ** l
    for a in range(D):
        for s in (-1, 1):
            nk = list(k)
            nk[a] = (nk[a] + s) % n
            if _covering_level(mesh, l, tuple(nk)) is not None:
                continue
            # the neighbour is split: its children next to the face must be leaves
            others = [b for b in range(D) if b != a]
            for t in range(2 ** (D - 1)):
                ck = [2 * x for x in nk]
                ck[a] += 1 if s < 0 else 0
                for j, b in enumerate(others):
                    ck[b] += (t >> j) & 1
                if _covering_level(mesh, l + 1, tuple(ck)) is None:
                    return False
    return True


def plan(leaves, D, refine, groups, coarsen):
    """New leaves and their sources, Morton-sorted: list of ((level, ijk), src)
    with src ('copy', c), ('prolong', c, o) or ('restrict', g)."""
    mesh = {}
    for c, (l, k) in enumerate(leaves):
        if refine[c]:
            for o in range(2 ** D):
                mesh[(l + 1, tuple(2 * k[a] + ((o >> a) & 1) for a in range(D)))] = ("prolong", c, o)
        else:
            mesh[(l, tuple(k))] = ("copy", c)
    # 2:1 balance by refinement of the coarser side (one level: sources stay copies)
    changed = True
    while changed:
        changed = False
        for (l, k), src in sorted(mesh.items()):
            if src[0] == "copy" and not _face_ok(mesh, l, k, D):
                del mesh[(l, k)]
                for o in range(2 ** D):
                    mesh[(l + 1, tuple(2 * k[a] + ((o >> a) & 1) for a in range(D)))] = ("prolong", src[1], o)
                changed = True
    # coarsening where the parent keeps the balance, repeated to a fixed point
    done = set()
    changed = True
    while changed:
        changed = False
        for g in coarsen:
            if g in done:
                continue
            pl, pk, mem = groups[g]
            keys = [(pl + 1, tuple(2 * pk[a] + ((o >> a) & 1) for a in range(D))) for o in range(2 ** D)]
            if not all(mesh.get(key) == ("copy", m) for key, m in zip(keys, mem)):
                continue
            trial = dict(mesh)
            for key in keys:
                del trial[key]
            trial[(pl, tuple(pk))] = ("restrict", g)
            if _face_ok(trial, pl, tuple(pk), D):
                mesh = trial
                done.add(g)
                changed = True
    items = list(mesh.items())
    lmax = max(l for (l, _), _ in items)
    def key(item):
        (l, k), _ = item
        kk = [x << (lmax - l) for x in k]
        z = 0
        for bit in range(lmax, -1, -1):
            for a in range(D - 1, -1, -1):
                z = (z << 1) | ((kk[a] >> bit) & 1)
        return (z, l)
    items.sort(key=key)
    return items


def remap(S, w, groups, items):
    """State [C_new, N] of the new leaves from the old state w [C, N]."""
    P, R = prolongation(S), restriction(S)
    out = np.zeros((len(items), w.shape[1]))
    for i, (_, src) in enumerate(items):
        if src[0] == "copy":
            out[i] = w[src[1]]
        elif src[0] == "prolong":
            out[i] = P[src[2]] @ w[src[1]]
        else:
            out[i] = np.einsum("oab,ob->a", R, w[groups[src[1]][2]])
    return out
