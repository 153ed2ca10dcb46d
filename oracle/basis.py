"""Exact-rational basis generator for the oracle (test infrastructure only).

This module is part of the CPU oracle. Only the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the GPU product path never
does. It shares no code with the CUDA library, which builds its own tables in
double precision from the same written conventions.

What it builds, each from the passage that defines it:

* univariate Legendre polynomials l_k with l_k(1) = 1 (Sec. 3.2, eq. legendre-3d);
* total-degree Legendre products P_k = l_k1 l_k2 (l_k3), k1+..+kD <= d,
  n(d) of them (Sec. 3.2; App. A for the 2D count);
* the locally divergence-free (LDF) vector basis (Sec. 3.3, App. A.2): curls of
  a pool of Legendre-product potentials of degree <= d+1, zero curls dropped,
  stable-sorted by total degree, then unnormalised Gram-Schmidt under the L2
  product of eq. innerp restricted to B; N_div = D n(d) - n(d-1) (eq. dimVdiv);
* the diagonal mass matrix M_l = <phi_l, phi_l> (eq. basis-ortho);
* Gauss-Legendre rules with d+1 points per dimension (Sec. 3.5), taken from
  numpy's leggauss (a library primitive) and pinned by exactness tests.

Conventions (the paper leaves them open, Sec. 3.2 "single integer"):
mode order = total degree ascending, then k1 descending, then k2 descending.
Pool order for LDF potentials = the same order over Legendre products of degree
1..d+1; in 3D each potential Q yields (Q,0,0), (0,Q,0), (0,0,Q) in the order
listed in App. A.2 (all x-potentials first, then y, then z).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import product
import numpy as np

# ---------------------------------------------------------------------------
# multivariate polynomials with Fraction coefficients: {exponent tuple: coeff}
# ---------------------------------------------------------------------------


def padd(a: dict, b: dict, s=1) -> dict:
    out = dict(a)
    for e, c in b.items():
        v = out.get(e, 0) + s * c
        if v == 0:
            out.pop(e, None)
        else:
            out[e] = v
    return out


def pscale(a: dict, s) -> dict:
    if s == 0:
        return {}
    return {e: c * s for e, c in a.items()}


def pmul(a: dict, b: dict) -> dict:
    out: dict = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            v = out.get(e, 0) + ca * cb
            if v == 0:
                out.pop(e, None)
            else:
                out[e] = v
    return out


def pderiv(a: dict, axis: int) -> dict:
    out = {}
    for e, c in a.items():
        k = e[axis]
        if k == 0:
            continue
        ne = list(e)
        ne[axis] = k - 1
        out[tuple(ne)] = out.get(tuple(ne), 0) + c * k
    return {e: c for e, c in out.items() if c != 0}


def pintegrate(a: dict) -> Fraction:
    """Exact integral over the reference cell [-1,1]^D."""
    tot = Fraction(0)
    for e, c in a.items():
        term = c
        for k in e:
            if k % 2:
                term = 0
                break
            term *= Fraction(2, k + 1)
        tot += term
    return tot


def pdegree(a: dict) -> int:
    return max((sum(e) for e in a), default=-1)


def peval(a: dict, pts: np.ndarray) -> np.ndarray:
    """Evaluate at points pts[..., D] in float64."""
    pts = np.asarray(pts, dtype=np.float64)
    out = np.zeros(pts.shape[:-1])
    for e, c in a.items():
        term = np.full(pts.shape[:-1], float(c))
        for ax, k in enumerate(e):
            if k:
                term = term * pts[..., ax] ** k
        out = out + term
    return out


# ---------------------------------------------------------------------------
# Legendre polynomials (Sec. 3.2)
# ---------------------------------------------------------------------------


@lru_cache(maxsize=None)
def legendre_1d(k: int) -> tuple:
    """Coefficients (c_0..c_k) of l_k, from Bonnet's recurrence
    (j+1) l_{j+1} = (2j+1) x l_j - j l_{j-1}; normalised so l_k(1) = 1."""
    if k == 0:
        return (Fraction(1),)
    prev, cur = [Fraction(1)], [Fraction(0), Fraction(1)]
    for j in range(1, k):
        nxt = [Fraction(0)] * (j + 2)
        for i, c in enumerate(cur):
            nxt[i + 1] += Fraction(2 * j + 1, j + 1) * c
        for i, c in enumerate(prev):
            nxt[i] -= Fraction(j, j + 1) * c
        prev, cur = cur, nxt
    return tuple(cur)


def n_modes(D: int, d: int) -> int:
    """n(d) of App. A: dimension of D-variate polynomials of degree <= d."""
    if d < 0:
        return 0
    if D == 2:
        return (d + 1) * (d + 2) // 2
    if D == 3:
        return (d + 1) * (d + 2) * (d + 3) // 6
    raise ValueError(D)


def n_div(D: int, d: int) -> int:
    """N_div = D n(d) - n(d-1), eq. dimVdiv."""
    return D * n_modes(D, d) - n_modes(D, d - 1)


def mode_list(D: int, d: int) -> list:
    """Multi-indices k with |k| <= d: total degree ascending, then k1
    descending, then k2 descending."""
    out = []
    for deg in range(d + 1):
        ks = [k for k in product(range(deg + 1), repeat=D) if sum(k) == deg]
        ks.sort(key=lambda k: tuple(-x for x in k))
        out.extend(ks)
    return out


def legendre_poly(k: tuple) -> dict:
    """P_k = prod_i l_{k_i}(xi_i) (eq. legendre-3d) as a D-variate polynomial."""
    D = len(k)
    poly = {tuple([0] * D): Fraction(1)}
    for ax, kk in enumerate(k):
        c1 = legendre_1d(kk)
        fac = {}
        for p, c in enumerate(c1):
            if c != 0:
                e = [0] * D
                e[ax] = p
                fac[tuple(e)] = c
        poly = pmul(poly, fac)
    return poly


def legendre_mass(k: tuple) -> Fraction:
    """<P_k, P_k> = prod 2/(2k_i+1)."""
    m = Fraction(1)
    for kk in k:
        m *= Fraction(2, 2 * kk + 1)
    return m


# ---------------------------------------------------------------------------
# locally divergence-free basis (Sec. 3.3, App. A.2)
# ---------------------------------------------------------------------------


def vdot(u: tuple, v: tuple) -> Fraction:
    """<u, v> = integral over [-1,1]^D of sum_a u_a v_a (eq. innerp on B)."""
    acc = {}
    for a, b in zip(u, v):
        if a and b:
            acc = padd(acc, pmul(a, b))
    return pintegrate(acc)


def vdiv(u: tuple) -> dict:
    acc = {}
    for ax, comp in enumerate(u):
        acc = padd(acc, pderiv(comp, ax))
    return acc


def _curls(D: int, Q: dict) -> list:
    if D == 2:
        # stream function Q: (dQ/dy, -dQ/dx)
        return [(pderiv(Q, 1), pscale(pderiv(Q, 0), -1))]
    # (Q,0,0) -> (0, dQ/dz, -dQ/dy); (0,Q,0) -> (-dQ/dz, 0, dQ/dx);
    # (0,0,Q) -> (dQ/dy, -dQ/dx, 0)
    return [
        ({}, pderiv(Q, 2), pscale(pderiv(Q, 1), -1)),
        (pscale(pderiv(Q, 2), -1), {}, pderiv(Q, 0)),
        (pderiv(Q, 1), pscale(pderiv(Q, 0), -1), {}),
    ]


def _vdeg(u: tuple) -> int:
    return max(pdegree(c) for c in u)


@lru_cache(maxsize=None)
def ldf_basis(D: int, d: int) -> tuple:
    """Orthogonal LDF basis of degree <= d as a tuple of D-component vector
    polynomials, sorted by total degree (App. A.2)."""
    pots = [legendre_poly(k) for k in mode_list(D, d + 1) if sum(k) >= 1]
    if D == 2:
        pool = [_curls(2, Q)[0] for Q in pots]
    else:
        per = [_curls(3, Q) for Q in pots]
        pool = [c[i] for i in range(3) for c in per]
    pool = [v for v in pool if any(v)]
    pool.sort(key=_vdeg)  # stable: keeps the pool order within a degree
    basis: list = []
    norms: list = []
    target = n_div(D, d)
    for v in pool:
        r = v
        for e, ee in zip(basis, norms):
            c = vdot(v, e) / ee
            if c != 0:
                r = tuple(padd(a, b, -c) for a, b in zip(r, e))
        if any(r):
            basis.append(r)
            norms.append(vdot(r, r))
        if len(basis) == target:
            break
    assert len(basis) == target, (len(basis), target)
    return tuple(basis)


def ldf_degrees(D: int, d: int) -> list:
    return [_vdeg(v) for v in ldf_basis(D, d)]


def ldf_mass(D: int, d: int) -> list:
    return [vdot(v, v) for v in ldf_basis(D, d)]


# ---------------------------------------------------------------------------
# Gauss-Legendre quadrature (Sec. 3.5): d+1 points per dimension
# ---------------------------------------------------------------------------


def gauss_1d(npts: int):
    x, w = np.polynomial.legendre.leggauss(npts)
    return x.astype(np.float64), w.astype(np.float64)


def gauss_tensor(D: int, npts: int):
    """Tensor Gauss rule on [-1,1]^D. Point order: last axis fastest."""
    x, w = gauss_1d(npts)
    grids = np.meshgrid(*([x] * D), indexing="ij")
    wg = np.meshgrid(*([w] * D), indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=-1)
    wts = np.prod(np.stack([g.reshape(-1) for g in wg], axis=-1), axis=-1)
    return pts, wts
