"""Pins of the Powell q^dagger of eq. powellq-interp (Sec. 4.1.3) and of the
HLLD interface state it uses: the closed form against the layer average of q
along the linear path in primitive variables, its reduction to q(u), the
interface state in the supersonic and contact cases, and the scheme's rhs
with both choices of q^dagger where B^n is continuous."""
import numpy as np

from oracle import basis as B
from oracle import mhd
from oracle.dg import Params, Scheme

G = 5.0 / 3.0


def test_interp_q_is_the_layer_average_along_the_linear_path():
    """(1/eps) int_layer q(u(s)) ds with v, B linear in s from (v_L, B_L) to
    (v_F, B_F): Gauss-Legendre in s (3 points: exact for the quadratic v.B)."""
    rng = np.random.default_rng(0)
    vL, BL, vF, BF = (rng.standard_normal((20, 3)) for _ in range(4))
    s, ws = B.gauss_1d(3)
    s, ws = 0.5 * (s + 1.0), 0.5 * ws
    avg = np.zeros((20, 8))
    for si, wi in zip(s, ws):
        v = vL + si * (vF - vL)
        Bf = BL + si * (BF - BL)
        avg[:, mhd.MX:mhd.MZ + 1] += wi * Bf
        avg[:, mhd.EN] += wi * np.sum(v * Bf, -1)
        avg[:, mhd.BX:mhd.BZ + 1] += wi * v
    assert np.abs(mhd.powell_q_interp(vL, BL, vF, BF) - avg).max() < 1e-14


def test_interp_q_reduces_to_q_of_the_state():
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.5, 2.0, 10)
    v = rng.standard_normal((10, 3))
    Bf = rng.standard_normal((10, 3))
    U = mhd.conserved(rho, v, rng.uniform(0.5, 2.0, 10), Bf, G)
    assert np.abs(mhd.powell_q_interp(v, Bf, v, Bf) - mhd.powell_q(U, G)).max() < 1e-13


def _hlld_state(rL, vL, pL, BL, rR, vR, pR, BR, axis=0):
    Bn = 0.5 * (BL[..., axis] + BR[..., axis])
    return mhd.hlld(rL, vL, pL, BL, rR, vR, pR, BR, Bn, axis, G, state=True)


def test_hlld_interface_state_supersonic_and_identical():
    """Supersonic flow: the upwind trace (B_n replaced by B^n_F); identical
    states: the state itself; the flux is unchanged by asking for the state."""
    one = np.ones(1)
    BL = np.array([[0.3, 0.2, -0.1]])
    BR = np.array([[0.3, -0.4, 0.5]])
    for sgn, up in ((1.0, "L"), (-1.0, "R")):
        vL = np.array([[sgn * 20.0, 0.1, 0.2]])
        vR = np.array([[sgn * 21.0, -0.3, 0.1]])
        F, vF, BF = _hlld_state(one, vL, one, BL, 2 * one, vR, 1.5 * one, BR)
        vu, Bu = (vL, BL) if up == "L" else (vR, BR)
        Bexp = Bu.copy()
        Bexp[0, 0] = 0.3
        assert np.allclose(vF, vu, atol=1e-14) and np.allclose(BF, Bexp, atol=1e-14)
        F0 = mhd.hlld(one, vL, one, BL, 2 * one, vR, 1.5 * one, BR, np.array([0.3]), 0, G)
        assert np.array_equal(F, F0)
    v = np.array([[0.3, -0.2, 0.1]])
    F, vF, BF = _hlld_state(one, v, one, BL, one, v, one, BL)
    assert np.allclose(vF, v, atol=1e-13) and np.allclose(BF, BL, atol=1e-13)


def test_hlld_interface_state_at_a_contact():
    """An isolated contact (only rho jumps) moving right: HLLD resolves it
    exactly, so the interface state is the left state."""
    one = np.ones(1)
    v = np.array([[0.4, 0.1, -0.2]])
    Bf = np.array([[0.5, 0.3, 0.2]])
    F, vF, BF = _hlld_state(one, v, one, Bf, 3 * one, v, one, Bf)
    assert np.allclose(vF, v, atol=1e-12) and np.allclose(BF, Bf, atol=1e-12)


def _cells(S, fn):
    return S.project(fn)


def test_rhs_with_interp_q_equals_mean_q_when_bn_is_continuous():
    """Uniform B, varying density, velocity and pressure: B^n is continuous at
    every face, so the Powell face term vanishes for either q^dagger; a jump in
    B_x across the x faces makes the two choices differ."""
    def smooth_b(x):
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])
        one = np.ones_like(rho)
        v = np.stack([0.2 * one, 0.1 * np.sin(2 * np.pi * x[..., 2]), 0.0 * one], -1)
        return mhd.conserved(rho, v, 1.0 + 0.1 * rho, np.stack([0.5 * one, 0.2 * one, 0.1 * one], -1), G)

    def kinked_b(x):
        u = smooth_b(x)
        u[..., mhd.BX] += 0.2 * np.abs(np.sin(np.pi * x[..., 0] * 3))   # B_x not in the LDF space per cell
        return u

    for fn, same in ((smooth_b, True), (kinked_b, False)):
        out = []
        for mode in ("mean", "interp"):
            S = Scheme(3, 2, "powell", G, 4, params=Params(powell_q=mode))
            out.append(S.rhs(_cells(S, fn)))
        diff = np.abs(out[0] - out[1]).max()
        assert (diff < 1e-12) if same else (diff > 1e-6)
