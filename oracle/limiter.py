"""Limiters of the oracle (test infrastructure only): Sec. 4.2 and 4.3.

* characteristic TVB slope limiter (Sec. 4.2.1 eq. tvb-limiter, Sec. 4.2.2):
  per direction a, the conserved degree-1 slopes u_xi and the mean differences
  D+ = (u_{a+} - u)/2, D- = (u - u_{a-})/2 (reference cell width 2) are mapped
  to characteristic variables with the left eigenvectors at the cell mean,
  limited field by field with
      sigma = u_xi                                  if |u_xi| <= M~ dx
            = minmod(u_xi, beta D+, beta D-)        otherwise,
  and marked triggered if |sigma - u_xi| > eps for some field. A triggered
  direction gets the slope R sigma; if any direction triggered, every weight of
  degree >= 2 is set to zero; cell means never change (Sec. 4.2.1).
* eigensystem: primitive variables W = (rho, v_n, v_t1, v_t2, p, B_t1, B_t2)
  with the Roe & Balsara (1996) normalised right eigenvectors of the seven MHD
  waves; the normal field B_n is a separate characteristic field -- the
  divergence wave of the 8-wave Powell system (Sec. 4.1.2), or with psi the
  pair (B_n, psi) of the linear GLM system with speeds -/+ c_h. Conserved slopes
  are converted with dW/dU at the mean; L = R^-1 (numpy inverse).
* LDF slope fix (Sec. 4.2.4): diagonal slopes rescaled by delta-/delta+ (or
  delta+/delta-), then the linear divergence-free field is projected exactly
  onto the LDF basis of degree <= 1.
* positivity limiter (Sec. 4.3): floors on the cell means with the injected
  mass and energy recorded, then tau_rho (eq. tau_rho) and, from the
  density-limited state, tau_p (eq. tau_press) over all volume and face Gauss
  points; w <- tau w + (1 - tau) w_mean (eq. wtilde).
"""
from __future__ import annotations

from fractions import Fraction
import numpy as np

from . import basis as B
from . import mhd

# --------------------------------------------------------------------- eigensystem


def _roe_balsara(rho, u, v, w, p, bn, bt1, bt2, gamma):
    """Right eigenvectors (columns) of the 7-wave primitive system along the
    normal, variables (rho, u, v, w, p, B_t1, B_t2), and the wave speeds."""
    a2 = gamma * p / rho
    sr = np.sqrt(rho)
    bt2sq = bt1 * bt1 + bt2 * bt2
    b2 = (bn * bn + bt2sq) / rho
    cax2 = bn * bn / rho
    disc = np.sqrt(max((a2 + b2) ** 2 - 4.0 * a2 * cax2, 0.0))
    cf2 = 0.5 * (a2 + b2 + disc)
    cs2 = max(0.5 * (a2 + b2 - disc), 0.0)
    cf, cs, ca = np.sqrt(cf2), np.sqrt(cs2), np.sqrt(cax2)
    a = np.sqrt(a2)
    if cf2 - cs2 > 1e-12 * cf2:
        af = np.sqrt(max(a2 - cs2, 0.0) / (cf2 - cs2))
        as_ = np.sqrt(max(cf2 - a2, 0.0) / (cf2 - cs2))
    else:
        af, as_ = 1.0, 0.0
    bt = np.sqrt(bt2sq)
    if bt > 1e-12 * np.sqrt(rho * cf2):
        by, bz = bt1 / bt, bt2 / bt
    else:
        by = bz = 1.0 / np.sqrt(2.0)
    S = 1.0 if bn >= 0.0 else -1.0
    R = np.zeros((7, 7))
    R[:, 0] = [rho * af, -af * cf, as_ * cs * by * S, as_ * cs * bz * S, rho * af * a2, as_ * sr * a * by,
               as_ * sr * a * bz]
    R[:, 1] = [0, 0, -bz, by, 0, -bz * S * sr, by * S * sr]
    R[:, 2] = [rho * as_, -as_ * cs, -af * cf * by * S, -af * cf * bz * S, rho * as_ * a2, -af * sr * a * by,
               -af * sr * a * bz]
    R[:, 3] = [1, 0, 0, 0, 0, 0, 0]
    R[:, 4] = [rho * as_, as_ * cs, af * cf * by * S, af * cf * bz * S, rho * as_ * a2, -af * sr * a * by,
               -af * sr * a * bz]
    R[:, 5] = [0, 0, -bz, by, 0, bz * S * sr, -by * S * sr]
    R[:, 6] = [rho * af, af * cf, -as_ * cs * by * S, -as_ * cs * bz * S, rho * af * a2, as_ * sr * a * by,
               as_ * sr * a * bz]
    lam = np.array([u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf])
    return R, lam


def dW_dU(U, gamma):
    """Jacobian of primitives (rho, v, p, B[, psi]) w.r.t. conserved variables."""
    nv = len(U)
    rho = U[0]
    v = U[1:4] / rho
    Bv = U[5:8]
    J = np.zeros((nv, nv))
    J[0, 0] = 1.0
    for i in range(3):
        J[1 + i, 0] = -v[i] / rho
        J[1 + i, 1 + i] = 1.0 / rho
    g1 = gamma - 1.0
    J[4, 0] = 0.5 * g1 * np.dot(v, v)
    J[4, 1:4] = -g1 * v
    J[4, 4] = g1
    J[4, 5:8] = -g1 * Bv
    for i in range(5, nv):
        J[i, i] = 1.0
    return J


def dU_dW(U, gamma):
    nv = len(U)
    rho = U[0]
    v = U[1:4] / rho
    Bv = U[5:8]
    J = np.zeros((nv, nv))
    J[0, 0] = 1.0
    for i in range(3):
        J[1 + i, 0] = v[i]
        J[1 + i, 1 + i] = rho
    J[4, 0] = 0.5 * np.dot(v, v)
    J[4, 1:4] = rho * v
    J[4, 4] = 1.0 / (gamma - 1.0)
    J[4, 5:8] = Bv
    for i in range(5, nv):
        J[i, i] = 1.0
    return J


def eigensystem(U, axis, gamma, ch=None):
    """(R, L, speeds) of the characteristic decomposition along `axis` in
    CONSERVED variables at state U (8 or 9 variables)."""
    nv = len(U)
    rho = U[0]
    vel = U[1:4] / rho
    Bv = U[5:8]
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * vel @ vel - 0.5 * Bv @ Bv)
    n, t1, t2 = axis, (axis + 1) % 3, (axis + 2) % 3
    R7, lam7 = _roe_balsara(rho, vel[n], vel[t1], vel[t2], p, Bv[n], Bv[t1], Bv[t2], gamma)
    # primitive index of each rotated 7-wave variable, then B_n (and psi)
    idx7 = [0, 1 + n, 1 + t1, 1 + t2, 4, 5 + t1, 5 + t2]
    RW = np.zeros((nv, nv))
    for i, pi in enumerate(idx7):
        RW[pi, :7] = R7[i]
    lam = list(lam7)
    if nv == 8:
        RW[5 + n, 7] = 1.0                 # divergence wave (Powell), speed v_n
        lam.append(vel[n])
    else:
        RW[5 + n, 7] = 1.0                 # GLM pair: (B_n, psi) = (1, -c_h), (1, +c_h)
        RW[8, 7] = -ch
        RW[5 + n, 8] = 1.0
        RW[8, 8] = ch
        lam += [-ch, ch]
    RU = dU_dW(U, gamma) @ RW
    LU = np.linalg.inv(RW) @ dW_dU(U, gamma)
    return RU, LU, np.array(lam)


# ---------------------------------------------------------------------- helpers


def minmod3(a, b, c):
    if a > 0 and b > 0 and c > 0:
        return min(a, b, c)
    if a < 0 and b < 0 and c < 0:
        return max(a, b, c)
    return 0.0


class Limiter:
    """Limiters for an oracle Scheme (uniform periodic mesh)."""

    def __init__(self, S, tvb=True, positivity=True):
        self.S = S
        self.tvb, self.pos = tvb, positivity
        D = S.D
        self.deg1 = [S.modes.index(tuple(1 if i == a else 0 for i in range(D))) for a in range(D)]
        self.mode_deg = [sum(k) for k in S.modes]
        if S.divb == "powell":
            ldf = S.ldf
            self.ldf_deg = B.ldf_degrees(D, S.d)
            # linear slope of LDF row j, component c, along a: <phi_jc, xi_a>/<xi_a, xi_a>
            xi = [{tuple(1 if i == a else 0 for i in range(D)): Fraction(1)} for a in range(D)]
            nrm = B.pintegrate(B.pmul(xi[0], xi[0]))
            self.ldf_slope = np.array([[[float(B.pintegrate(B.pmul(comp, xi[a])) / nrm) if comp else 0.0
                                         for a in range(D)] for comp in ldf[j]] for j in range(len(ldf))])
            self.ldf_mean = np.array([[float(B.pintegrate(comp) / 2 ** D) if comp else 0.0 for comp in ldf[j]]
                                      for j in range(len(ldf))])
            # exact projection of the linear field xi_a e_c onto LDF rows of degree <= 1
            self.low = [j for j in range(len(ldf)) if self.ldf_deg[j] <= 1]
            lin = np.zeros((len(ldf), D, D))  # [j, c, a]: <phi_j, xi_a e_c> / M_j
            const = np.zeros((len(ldf), D))
            for j in range(len(ldf)):
                Mj = B.vdot(ldf[j], ldf[j])
                for c in range(D):
                    comp = ldf[j][c]
                    if not comp:
                        continue
                    const[j, c] = float(B.pintegrate(comp) / Mj)
                    for a in range(D):
                        lin[j, c, a] = float(B.pintegrate(B.pmul(comp, xi[a])) / Mj)
            self.proj_lin, self.proj_const = lin, const
        # all volume and face Gauss points for positivity (Sec. 4.3)
        pts = [S.Sv]
        for a in range(D):
            for s in (-1, 1):
                pts.append(S.Sf[(a, s)])
        self.Spos = np.concatenate(pts, axis=1)
        self.injected = np.zeros(2)  # mass, energy added by the mean floors

    # ----------------------------------------------------- conserved slopes
    def slopes(self, w):
        """u_xi[cell, a, var]: degree-1 coefficient along a of every variable."""
        S = self.S
        out = np.zeros((S.C, S.D, S.V))
        for r, (kind, v, i) in enumerate(S.rows):
            if kind == "L" and self.mode_deg[i] == 1:
                a = self.deg1.index(i)
                out[:, a, v] += w[:, r]
            elif kind == "B":
                for c in range(S.D):
                    for a in range(S.D):
                        if self.ldf_slope[i, c, a] != 0.0:
                            out[:, a, mhd.BX + c] += w[:, r] * self.ldf_slope[i, c, a]
        return out

    # ----------------------------------------------------- neighbour differences
    def mean_differences(self, m):
        """D+[c, a], D-[c, a]: mean differences per direction in units of the
        reference half-width. Uniform mesh: (u_{a+} - u)/2 and (u - u_{a-})/2.
        Octree (reading of Sec. 4.4, which defers to Schaal et al. 2015): the
        neighbour mean (the average of the adjacent finer leaves when refined)
        divided by the centre distance in units of dx_K/2: 2 same level, 3 for
        a coarser neighbour, 1.5 for finer ones."""
        S = self.S
        if not hasattr(S, "faces"):
            dp = np.stack([0.5 * (m[S.nbr_plus[a]] - m) for a in range(S.D)], 1)
            dm = np.stack([0.5 * (m - m[S.nbr_minus[a]]) for a in range(S.D)], 1)
            return dp, dm
        C, D, V = S.C, S.D, m.shape[1]
        acc = np.zeros((C, D, 2, V))
        cnt = np.zeros((C, D, 2))
        fac = np.zeros((C, D, 2))
        for cL, cR, a, kind, sub in S.faces:
            # cR sees cL on its -a side; cL sees cR on its +a side
            for cell, nb, side in ((cR, cL, 0), (cL, cR, 1)):
                acc[cell, a, side] += m[nb]
                cnt[cell, a, side] += 1
                if kind == 0:
                    f = 2.0
                elif (kind == 1 and cell == cL) or (kind == 2 and cell == cR):
                    f = 1.5          # this cell is coarse: finer neighbours
                else:
                    f = 3.0          # the neighbour is coarse
                fac[cell, a, side] = f
        nbm = acc / cnt[..., None]
        dp = (nbm[:, :, 1] - m[:, None, :]) / fac[:, :, 1, None]
        dm = (m[:, None, :] - nbm[:, :, 0]) / fac[:, :, 0, None]
        return dp, dm

    # ----------------------------------------------------- TVB-characteristic
    def tvb_limit(self, w, ch=None):
        S, P = self.S, self.S.P
        m = S.means(w)
        sl = self.slopes(w)
        out = w.copy()
        troubled = np.zeros(S.C, dtype=bool)
        dpa, dma = self.mean_differences(m)
        dxc = S.dxc if hasattr(S, "dxc") else np.full(S.C, S.dx)
        for c in range(S.C):
            thr = P.Mtilde * dxc[c]
            new_sl = sl[c].copy()
            hit = False
            for a in range(S.D):
                dp = dpa[c, a]
                dm = dma[c, a]
                R, L, _ = eigensystem(m[c], a, S.gamma, ch)
                cx, cp, cm = L @ sl[c, a], L @ dp, L @ dm
                sig = cx.copy()
                trig = False
                for k in range(S.V):
                    if abs(cx[k]) > thr:
                        sig[k] = minmod3(cx[k], P.beta * cp[k], P.beta * cm[k])
                    if abs(sig[k] - cx[k]) > P.tvb_eps:
                        trig = True
                if trig:
                    new_sl[a] = R @ sig
                    hit = True
            if not hit:
                continue
            troubled[c] = True
            self._assign(out, c, m[c], new_sl)
        return out, troubled

    def _assign(self, out, c, mean, new_sl):
        """Write limited degree-1 slopes, zero degree >= 2, keep means."""
        S = self.S
        for r, (kind, v, i) in enumerate(S.rows):
            if kind == "L":
                dgr = self.mode_deg[i]
                if dgr == 1:
                    out[c, r] = new_sl[self.deg1.index(i), v]
                elif dgr >= 2:
                    out[c, r] = 0.0
        if S.divb == "powell":
            D = S.D
            Bs = np.array([[new_sl[a, mhd.BX + cc] for a in range(D)] for cc in range(D)])  # [c, a]
            diag = np.array([Bs[k, k] for k in range(D)])
            dsum = diag.sum()
            dpos = np.sum(np.maximum(diag, 0.0))
            dneg = np.sum(np.maximum(-diag, 0.0))
            if dsum > 0:
                fac = dneg / dpos
                diag = np.where(diag > 0, fac * diag, diag)
            elif dsum < 0:
                fac = dpos / dneg
                diag = np.where(diag < 0, fac * diag, diag)
            for k in range(D):
                Bs[k, k] = diag[k]
            Bmean = mean[mhd.BX:mhd.BX + D]
            ldf0 = 5 * S.n
            for j in range(len(S.ldf)):
                r = ldf0 + j
                if self.ldf_deg[j] > 1:
                    out[c, r] = 0.0
                    continue
                val = 0.0
                for cc in range(D):
                    val += self.proj_const[j, cc] * Bmean[cc]
                    for a in range(D):
                        val += self.proj_lin[j, cc, a] * Bs[cc, a]
                out[c, r] = val

    # ----------------------------------------------------- positivity
    def positivity(self, w):
        S, P = self.S, self.S.P
        g = S.gamma
        out = w.copy()
        is_mean = S.is_mean
        m = S.means(out)
        for c in range(S.C):
            rho_b = m[c, mhd.RHO]
            if rho_b < P.eps_rho:
                r0 = S.rows.index(("L", mhd.RHO, 0))
                self.injected[0] += (P.eps_rho - rho_b) * S.dx ** S.D
                out[c, r0] = P.eps_rho
                m[c, mhd.RHO] = P.eps_rho
            pb = mhd.primitives(m[c], g)[2]
            if pb < P.eps_p:
                rE = S.rows.index(("L", mhd.EN, 0))
                dE = (P.eps_p - pb) / (g - 1.0)
                self.injected[1] += dE * S.dx ** S.D
                out[c, rE] += dE
                m[c, mhd.EN] += dE
        u = np.einsum("cr,rqv->cqv", out, self.Spos)
        for c in range(S.C):
            rho_b = m[c, mhd.RHO]
            rq = u[c, :, mhd.RHO]
            bad = rq < P.eps_rho
            tau = 1.0
            if np.any(bad):
                tau = min(1.0, np.min((rho_b - P.eps_rho) / (rho_b - rq[bad])))
            if tau < 1.0:
                out[c, ~is_mean] *= tau
        u = np.einsum("cr,rqv->cqv", out, self.Spos)
        for c in range(S.C):
            pb = mhd.primitives(m[c], g)[2]
            pq = mhd.primitives(u[c], g)[2]
            bad = pq < P.eps_p
            tau = 1.0
            if np.any(bad):
                tau = min(1.0, np.min((pb - P.eps_p) / (pb - pq[bad])))
            if tau < 1.0:
                out[c, ~is_mean] *= tau
        return out

    def __call__(self, w, ch=None):
        if self.tvb:
            w, _ = self.tvb_limit(w, ch)
        if self.pos:
            w = self.positivity(w)
        return w
