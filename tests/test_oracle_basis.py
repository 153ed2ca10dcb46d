"""Pins of the oracle's basis and quadrature against what the paper and the
mathematics fix (no GPU)."""
import os
from collections import Counter
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import basis as B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_exactness(n):
    # Sec. 3.5: n points integrate degree <= 2n-1 exactly
    x, w = B.gauss_1d(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # and not degree 2n
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


def test_gauss_closed_forms():
    x, w = B.gauss_1d(1)
    assert x[0] == 0.0 and w[0] == 2.0
    x, w = B.gauss_1d(2)
    assert np.allclose(sorted(x), [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    x, w = B.gauss_1d(3)
    assert np.allclose(sorted(x), [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(sorted(w), [5 / 9, 5 / 9, 8 / 9], atol=1e-15)


def test_legendre_1d_textbook():
    F = Fraction
    assert B.legendre_1d(2) == (F(-1, 2), F(0), F(3, 2))
    assert B.legendre_1d(3) == (F(0), F(-3, 2), F(0), F(5, 2))
    assert B.legendre_1d(4) == (F(3, 8), F(0), F(-30, 8), F(0), F(35, 8))
    for k in range(6):
        assert sum(B.legendre_1d(k)) == 1  # l_k(1) = 1


@pytest.mark.parametrize("D,d", [(2, 3), (3, 2)])
def test_legendre_orthogonality(D, d):
    modes = B.mode_list(D, d)
    assert len(modes) == B.n_modes(D, d)
    polys = [B.legendre_poly(k) for k in modes]
    for i, (ki, pi) in enumerate(zip(modes, polys)):
        for j in range(i, len(modes)):
            ip = B.pintegrate(B.pmul(pi, polys[j]))
            if i == j:
                assert ip == B.legendre_mass(ki)
            else:
                assert ip == 0


def test_ndiv_table_a1():
    for D, d, nd in _rows("table_a1_ndiv.txt"):
        D, d, nd = int(D), int(d), int(nd)
        assert B.n_div(D, d) == nd
        if d <= (4 if D == 2 else 3):
            assert len(B.ldf_basis(D, d)) == nd


def test_dof_counts_fig1_fig2_and_sec5():
    # Fig. 1: 3D d=1 -> N = 5 n(1) + N_div = 20 + 11 = 31 ; Fig. 2: 2D d=1 -> 23
    assert 5 * B.n_modes(3, 1) + B.n_div(3, 1) == 31
    assert 6 * B.n_modes(2, 1) + B.n_div(2, 1) == 23
    # Sec. 5.4 N_DoF for 2D Powell: DG-2 128^2 ~ 3.8e5, DG-2 256^2 ~ 1.5e6, DG-3 128^2 ~ 7.4e5
    per = lambda d: 6 * B.n_modes(2, d) + B.n_div(2, d)
    assert round(per(1) * 128 ** 2 / 1e4) == 38
    assert round(per(1) * 256 ** 2 / 1e5) == 15
    assert round(per(2) * 128 ** 2 / 1e4) == 74


@pytest.mark.parametrize("D,d", [(2, 3), (3, 2)])
def test_ldf_divergence_free_and_orthogonal(D, d):
    basis = B.ldf_basis(D, d)
    for v in basis:
        assert B.vdiv(v) == {}
        assert B.pdegree(B.vdiv(v)) == -1
    for i in range(len(basis)):
        for j in range(i + 1, len(basis)):
            assert B.vdot(basis[i], basis[j]) == 0
        assert B.vdot(basis[i], basis[i]) > 0
    degs = B.ldf_degrees(D, d)
    assert degs == sorted(degs)
    # block sizes: N_div(k) - N_div(k-1) vectors of degree exactly k
    cnt = Counter(degs)
    for k in range(d + 1):
        assert cnt[k] == B.n_div(D, k) - (B.n_div(D, k - 1) if k else 0)


def test_ldf_spans_all_divfree_polynomials():
    # every divergence-free linear field lies in the degree-1 span (exact projection)
    D, d = 3, 2
    basis = B.ldf_basis(D, d)
    F = Fraction
    # u = (x + 2y, 3z - y, x - 0... ) with div = 1 - 1 + 0 = 0
    u = ({(1, 0, 0): F(1), (0, 1, 0): F(2)}, {(0, 0, 1): F(3), (0, 1, 0): F(-1)}, {(1, 0, 0): F(1)})
    assert B.vdiv(u) == {}
    rec = ({}, {}, {})
    for v in basis:
        c = B.vdot(u, v) / B.vdot(v, v)
        rec = tuple(B.padd(a, B.pscale(b, c)) for a, b in zip(rec, v))
    for a, b in zip(rec, u):
        assert B.padd(a, b, -1) == {}


def test_table_b1_ldf_projection_contamination():
    basis = B.ldf_basis(2, 5)
    degs = B.ldf_degrees(2, 5)
    ux = ({(1, 0): Fraction(1)}, {})
    uy = ({}, {(0, 1): Fraction(1)})
    got = Counter()
    for v, k in zip(basis, degs):
        pa, pb = B.vdot(ux, v), B.vdot(uy, v)
        if pa or pb:
            got[(k, pa, pb)] += 1
    want = Counter((int(k), Fraction(a), Fraction(b)) for k, a, b in _rows("table_b1_ldf_projection.txt"))
    assert got == want
    assert len(basis) == 27
