"""Pointwise ideal-MHD physics for the oracle (test infrastructure only).

Plain FP64 numpy, vectorised over leading axes; the last axis holds the
conserved variables (rho, m_x, m_y, m_z, E, B_x, B_y, B_z[, psi]).
Only tests, the smoke check and the benchmark's CPU-baseline leg may use it.

* conserved variables and EOS: Sec. 2, eqs. cns-vec and the gamma law;
* analytic fluxes: eq. mhd-flux; GLM additions (psi I in the B flux, c_h^2 B
  as the psi flux): Sec. 4.1.5, eqs. dedner-induction / dedner-psi-evol;
* face normal field B^n_F: Sec. 4.1.3, eq. bxface-average-alfven;
* GLM interface values psi*, B_n*: upwinding of the linear 2x2 GLM system
  (Sec. 4.1.5, following Dedner et al. 2002);
* HLLD: the five-wave flux of Miyoshi & Kusano (2005) used everywhere
  (Sec. 4.1.2). The paper does not print it; this follows the published
  method (outer speeds, S_M, p_T*, starred and double-starred states).
"""
from __future__ import annotations

import numpy as np

RHO, MX, MY, MZ, EN, BX, BY, BZ, PSI = range(9)


def primitives(U, gamma):
    """(rho, v[...,3], p, B[...,3]) from conserved U (Sec. 2)."""
    rho = U[..., RHO]
    v = U[..., MX:MZ + 1] / rho[..., None]
    B = U[..., BX:BZ + 1]
    kin = 0.5 * rho * np.sum(v * v, axis=-1)
    mag = 0.5 * np.sum(B * B, axis=-1)
    p = (gamma - 1.0) * (U[..., EN] - kin - mag)
    return rho, v, p, B


def conserved(rho, v, p, B, gamma, psi=None):
    nv = 8 if psi is None else 9
    U = np.zeros(rho.shape + (nv,))
    U[..., RHO] = rho
    U[..., MX:MZ + 1] = rho[..., None] * v
    U[..., EN] = p / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, -1) + 0.5 * np.sum(B * B, -1)
    U[..., BX:BZ + 1] = B
    if psi is not None:
        U[..., PSI] = psi
    return U


def flux(U, axis, gamma, ch2=None):
    """Analytic flux f_axis(U), eq. mhd-flux; with ch2 (= c_h^2) given, the
    GLM flux of Sec. 4.1.5 (extra psi on the B_axis row, c_h^2 B_axis for psi)."""
    rho, v, p, B = primitives(U, gamma)
    pT = p + 0.5 * np.sum(B * B, -1)
    va = v[..., axis]
    Ba = B[..., axis]
    vB = np.sum(v * B, -1)
    F = np.zeros_like(U)
    F[..., RHO] = U[..., MX + axis]
    for i in range(3):
        F[..., MX + i] = U[..., MX + i] * va - B[..., i] * Ba
        F[..., BX + i] = B[..., i] * va - v[..., i] * Ba
    F[..., MX + axis] += pT
    F[..., EN] = (U[..., EN] + pT) * va - vB * Ba
    if ch2 is not None:
        psi = U[..., PSI]
        F[..., BX + axis] += psi
        F[..., PSI] = ch2 * Ba
    return F


def fast_speed(rho, p, B, Bn, gamma):
    """Fast magnetosonic speed along a direction with normal field Bn."""
    a2 = gamma * p / rho
    b2 = np.sum(B * B, -1) / rho
    bn2 = Bn * Bn / rho
    disc = np.maximum((a2 + b2) ** 2 - 4.0 * a2 * bn2, 0.0)
    return np.sqrt(0.5 * (a2 + b2 + np.sqrt(disc)))


def bn_face(rhoL, rhoR, BnL, BnR):
    """B^n_F, eq. bxface-average-alfven: average weighted by 1/sqrt(rho)."""
    sL = 1.0 / np.sqrt(rhoL)
    sR = 1.0 / np.sqrt(rhoR)
    return (BnL * sL + BnR * sR) / (sL + sR)


def glm_face(BnL, BnR, psiL, psiR, ch):
    """Upwinded interface values (B_n*, psi*) of the linear GLM subsystem
    dB_n/dt + dpsi/dx = 0, dpsi/dt + c_h^2 dB_n/dx = 0 (Dedner et al. 2002)."""
    bstar = 0.5 * (BnL + BnR) - (psiR - psiL) / (2.0 * ch)
    pstar = 0.5 * (psiL + psiR) - 0.5 * ch * (BnR - BnL)
    return bstar, pstar


def _rot(axis):
    """Permutation (n, t1, t2) of spatial axes for a face normal to `axis`."""
    return axis, (axis + 1) % 3, (axis + 2) % 3


def hlld(rhoL, vL, pL, BL, rhoR, vR, pR, BR, Bn, axis, gamma, eps=1e-8, state=False):
    """HLLD flux (Miyoshi & Kusano 2005) across a face normal to `axis`, with
    the normal field of both states set to Bn beforehand (Sec. 4.1.3:
    primitives rho, v, p are kept, B_n := B^n_F).

    Returns the 8-component flux in the (x, y, z) frame; its B_axis entry is 0.
    With state=True also (v_F, B_F): velocity and field of the interface state
    u_F, the state of the Riemann fan that contains the interface (Sec. 4.1.3,
    "Interface state"), in the (x, y, z) frame.
    """
    n, t1, t2 = _rot(axis)
    shape = np.broadcast(rhoL, rhoR).shape

    def unpack(rho, v, p, B):
        u, vt, wt = v[..., n], v[..., t1], v[..., t2]
        By, Bz = B[..., t1], B[..., t2]
        Bsq = Bn * Bn + By * By + Bz * Bz
        E = p / (gamma - 1.0) + 0.5 * rho * (u * u + vt * vt + wt * wt) + 0.5 * Bsq
        pT = p + 0.5 * Bsq
        return u, vt, wt, By, Bz, E, pT

    uL, vtL, wtL, ByL, BzL, EL, pTL = unpack(rhoL, vL, pL, BL)
    uR, vtR, wtR, ByR, BzR, ER, pTR = unpack(rhoR, vR, pR, BR)

    def fstate(rho, u, vt, wt, By, Bz, E, pT):
        """Rotated-frame conserved state and flux (rho, m_n, m_t1, m_t2, E, B_n, B_t1, B_t2)."""
        U = np.stack([rho, rho * u, rho * vt, rho * wt, E, np.broadcast_to(Bn, rho.shape), By, Bz], -1)
        vB = u * Bn + vt * By + wt * Bz
        F = np.stack([
            rho * u,
            rho * u * u + pT - Bn * Bn,
            rho * vt * u - Bn * By,
            rho * wt * u - Bn * Bz,
            (E + pT) * u - Bn * vB,
            np.zeros(rho.shape),
            By * u - Bn * vt,
            Bz * u - Bn * wt,
        ], -1)
        return U, F

    BLs = BL.copy()
    BLs[..., n] = Bn
    BRs = BR.copy()
    BRs[..., n] = Bn
    cfL = fast_speed(rhoL, pL, BLs, Bn, gamma)
    cfR = fast_speed(rhoR, pR, BRs, Bn, gamma)
    cmax = np.maximum(cfL, cfR)
    SL = np.minimum(uL, uR) - cmax
    SR = np.maximum(uL, uR) + cmax

    dL = SL - uL
    dR = SR - uR
    den = dR * rhoR - dL * rhoL
    SM = (dR * rhoR * uR - dL * rhoL * uL - pTR + pTL) / den
    pTs = (dR * rhoR * pTL - dL * rhoL * pTR + rhoL * rhoR * dR * dL * (uR - uL)) / den

    def star(rho, u, vt, wt, By, Bz, E, pT, S, d):
        rs = rho * d / (S - SM)
        dd = rho * d * (S - SM) - Bn * Bn
        degen = np.abs(dd) < eps * (np.abs(rho * d * (S - SM)) + Bn * Bn)
        dds = np.where(degen, 1.0, dd)
        fac_v = Bn * (SM - u) / dds
        fac_b = (rho * d * d - Bn * Bn) / dds
        vts = np.where(degen, vt, vt - By * fac_v)
        wts = np.where(degen, wt, wt - Bz * fac_v)
        Bys = np.where(degen, By, By * fac_b)
        Bzs = np.where(degen, Bz, Bz * fac_b)
        vB = u * Bn + vt * By + wt * Bz
        vBs = SM * Bn + vts * Bys + wts * Bzs
        Es = (d * E - pT * u + pTs * SM + Bn * (vB - vBs)) / (S - SM)
        return rs, vts, wts, Bys, Bzs, Es

    rsL, vtsL, wtsL, BysL, BzsL, EsL = star(rhoL, uL, vtL, wtL, ByL, BzL, EL, pTL, SL, dL)
    rsR, vtsR, wtsR, BysR, BzsR, EsR = star(rhoR, uR, vtR, wtR, ByR, BzR, ER, pTR, SR, dR)

    sqL = np.sqrt(rsL)
    sqR = np.sqrt(rsR)
    sgn = np.where(Bn >= 0.0, 1.0, -1.0)
    SsL = SM - np.abs(Bn) / sqL
    SsR = SM + np.abs(Bn) / sqR
    inv = 1.0 / (sqL + sqR)
    vss = (sqL * vtsL + sqR * vtsR + (BysR - BysL) * sgn) * inv
    wss = (sqL * wtsL + sqR * wtsR + (BzsR - BzsL) * sgn) * inv
    Byss = (sqL * BysR + sqR * BysL + sqL * sqR * (vtsR - vtsL) * sgn) * inv
    Bzss = (sqL * BzsR + sqR * BzsL + sqL * sqR * (wtsR - wtsL) * sgn) * inv
    vBss = SM * Bn + vss * Byss + wss * Bzss
    vBsL = SM * Bn + vtsL * BysL + wtsL * BzsL
    vBsR = SM * Bn + vtsR * BysR + wtsR * BzsR
    EssL = EsL - sqL * (vBsL - vBss) * sgn
    EssR = EsR + sqR * (vBsR - vBss) * sgn

    UL, FL = fstate(rhoL, uL, vtL, wtL, ByL, BzL, EL, pTL)
    UR, FR = fstate(rhoR, uR, vtR, wtR, ByR, BzR, ER, pTR)

    def ustate(rs, vt, wt, By, Bz, E):
        return np.stack([rs, rs * SM, rs * vt, rs * wt, E, np.broadcast_to(Bn, rs.shape), By, Bz], -1)

    UsL = ustate(rsL, vtsL, wtsL, BysL, BzsL, EsL)
    UsR = ustate(rsR, vtsR, wtsR, BysR, BzsR, EsR)
    UssL = ustate(rsL, vss, wss, Byss, Bzss, EssL)
    UssR = ustate(rsR, vss, wss, Byss, Bzss, EssR)
    FsL = FL + SL[..., None] * (UsL - UL)
    FsR = FR + SR[..., None] * (UsR - UR)
    FssL = FsL + SsL[..., None] * (UssL - UsL)
    FssR = FsR + SsR[..., None] * (UssR - UsR)

    Fr = np.where((SL > 0)[..., None], FL,
         np.where((SsL >= 0)[..., None], FsL,
         np.where((SM >= 0)[..., None], FssL,
         np.where((SsR >= 0)[..., None], FssR,
         np.where((SR >= 0)[..., None], FsR, FR)))))
    if state:
        # region of the fan containing x/t = 0 (the selection of the flux above):
        # rotated (v_n, v_t1, v_t2, B_t1, B_t2) of that state; B_n = Bn throughout
        def pick(*vals):
            conds = [SL > 0, SsL >= 0, SM >= 0, SsR >= 0, SR >= 0]
            out = vals[5]
            for c, v in zip(reversed(conds), reversed(vals[:5])):
                out = np.where(c, v, out)
            return out
        smv = np.broadcast_to(SM, shape)
        vn = pick(uL, smv, smv, smv, smv, uR)
        vt = pick(vtL, vtsL, vss, vss, vtsR, vtR)
        wt = pick(wtL, wtsL, wss, wss, wtsR, wtR)
        By = pick(ByL, BysL, Byss, Byss, BysR, ByR)
        Bz = pick(BzL, BzsL, Bzss, Bzss, BzsR, BzR)
        vF = np.zeros(shape + (3,))
        BF = np.zeros(shape + (3,))
        vF[..., n], vF[..., t1], vF[..., t2] = vn, vt, wt
        BF[..., n], BF[..., t1], BF[..., t2] = np.broadcast_to(Bn, shape), By, Bz
    # rotate back: rotated index k -> xyz component
    F = np.zeros(shape + (8,))
    F[..., RHO] = Fr[..., 0]
    F[..., MX + n] = Fr[..., 1]
    F[..., MX + t1] = Fr[..., 2]
    F[..., MX + t2] = Fr[..., 3]
    F[..., EN] = Fr[..., 4]
    F[..., BX + n] = Fr[..., 5]
    F[..., BX + t1] = Fr[..., 6]
    F[..., BX + t2] = Fr[..., 7]
    if state:
        return F, vF, BF
    return F


def powell_q(U, gamma):
    """q(u) = (0, B, v.B, v), eq. powell-q, as a vector over the 8 MHD variables."""
    rho, v, p, B = primitives(U, gamma)
    q = np.zeros(U.shape[:-1] + (8,))
    q[..., MX:MZ + 1] = B
    q[..., EN] = np.sum(v * B, -1)
    q[..., BX:BZ + 1] = v
    return q


def powell_q_interp(vL, BL, vF, BF):
    """q^dagger of eq. powellq-interp: the Powell q of a state interpolated
    linearly in primitive variables between the trace u_L and the interface
    state u_F, averaged over the layer: (0, (B_L+B_F)/2,
    (2 B_L.v_L + B_L.v_F + B_F.v_L + 2 B_F.v_F)/6, (v_L+v_F)/2)."""
    q = np.zeros(np.broadcast(vL, vF).shape[:-1] + (8,))
    q[..., MX:MZ + 1] = 0.5 * (BL + BF)
    q[..., EN] = (2 * np.sum(BL * vL, -1) + np.sum(BL * vF, -1) + np.sum(BF * vL, -1)
                  + 2 * np.sum(BF * vF, -1)) / 6.0
    q[..., BX:BZ + 1] = 0.5 * (vL + vF)
    return q


def signal_speed(U, gamma):
    """c = sqrt(c_s^2 + c_A^2) (Sec. 3.6), an upper bound of the fast speed."""
    rho, v, p, B = primitives(U, gamma)
    return np.sqrt(gamma * p / rho + np.sum(B * B, -1) / rho)
