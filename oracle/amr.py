"""Oracle of the DG-MHD operator on a static octree AMR mesh (test
infrastructure only; Sec. 4.4 and the surface integral of eq. wdot).

Leaves are cubes (level l, integer coordinates k at that level) of a periodic
box of side L; level l has cell size L / 2^l. Faces, with 2:1 balance across
faces (one level difference at most):
* same level: one face per pair, integrated at the face's Gauss points;
* coarse-fine: one face per fine cell side; integrated at the FINE face's Gauss
  points. The fine side uses its own reference face; the coarse side sees the
  same physical points at reference coordinates xi_t = (xi_t,fine +/- 1)/2 on
  its own face, and its reference face measure is 1/4 of the fine one, so its
  quadrature weights are w_p / 4 (in 2D: 1/2). The flux F* is computed once per
  point and used by both sides, so the scheme stays conservative.
Each cell uses its own metric 2/dx_K (eq. wdot) and its own dx_K in eq. cfl.
The Powell face term of eq. powell-src-face uses each side's own trace.

Reuses the uniform oracle's basis, pointwise physics and state layout.
"""
from __future__ import annotations

import numpy as np

from . import basis as B
from . import mhd
from .dg import Scheme, Params


def balanced(leaves, D):
    """True if every leaf's face neighbours differ by at most one level."""
    S = {(l,) + tuple(k) for l, k in leaves}
    for l, k in leaves:
        n = 2 ** l
        for a in range(D):
            for s in (-1, 1):
                kk = list(k)
                kk[a] = (kk[a] + s) % n
                if (l,) + tuple(kk) in S:
                    continue
                if l > 0 and (l - 1,) + tuple(x // 2 for x in kk) in S:
                    continue
                # refined neighbour: its adjacent children must be leaves
                kids = []
                base = [2 * x for x in kk]
                ok = True
                for t in range(2 ** (D - 1)):
                    ch = list(base)
                    ch[a] += 1 if s < 0 else 0
                    others = [b for b in range(D) if b != a]
                    for j, b in enumerate(others):
                        ch[b] += (t >> j) & 1
                    if (l + 1,) + tuple(ch) not in S:
                        ok = False
                if not ok:
                    return False
    return True


class AMRScheme(Scheme):
    """Scheme on a leaf list [(level, (i, j[, k]))]. Cell order = list order."""

    def __init__(self, D, d, divb, gamma, leaves, L=1.0, params: Params | None = None):
        self.leaves = [(int(l), tuple(int(x) for x in k)) for l, k in leaves]
        self.D_ = D
        super().__init__(D, d, divb, gamma, 1, L=L, params=params)

    # ------------------------------------------------------------------ mesh
    def _build_mesh(self):
        D, L = self.D, self.L
        self.C = len(self.leaves)
        idx = {(l,) + k: c for c, (l, k) in enumerate(self.leaves)}
        self.level = np.array([l for l, _ in self.leaves])
        self.dxc = L / 2.0 ** self.level
        self.centers = np.array([[(k[a] + 0.5) * L / 2 ** l for a in range(D)] for l, k in self.leaves])
        # face records: (cL, cR, axis, kind, sub); kind 0 same level, 1 L coarse, 2 R coarse
        faces = []
        for c, (l, k) in enumerate(self.leaves):
            n = 2 ** l
            for a in range(D):
                others = [b for b in range(D) if b != a]
                for s in (-1, 1):
                    kk = list(k)
                    kk[a] = (kk[a] + s) % n
                    key = (l,) + tuple(kk)
                    if key in idx:
                        if s < 0:
                            faces.append((idx[key], c, a, 0, 0))
                        continue
                    pkey = (l - 1,) + tuple(x // 2 for x in kk)
                    if l > 0 and pkey in idx:
                        sub = sum(((k[b] & 1) << j) for j, b in enumerate(others))
                        if s < 0:
                            faces.append((idx[pkey], c, a, 1, sub))   # coarse on the left
                        else:
                            faces.append((c, idx[pkey], a, 2, sub))   # coarse on the right
                        continue
                    # finer neighbour: recorded from the fine side
        self.faces = faces
        self.ncell = (self.C,)
        self.dx = float(np.min(self.dxc))

    # --------------------------------------------------------------- tables
    def _sub_points(self, axis, side, sub):
        """Coarse-side reference points of sub-face `sub` on face (axis, side)."""
        pts, wf = self.face_points(axis, side)
        others = [b for b in range(self.D) if b != axis]
        out = pts.copy()
        for j, b in enumerate(others):
            bit = (sub >> j) & 1
            out[:, b] = 0.5 * (pts[:, b] + (1.0 if bit else -1.0))
        return out

    def _build_tables(self):
        super()._build_tables()
        self.Ssub = {}
        for a in range(self.D):
            for s in (-1, 1):
                for sub in range(2 ** (self.D - 1)):
                    self.Ssub[(a, s, sub)] = self.synth(self._sub_points(a, s, sub))
        self.sub_w = 1.0 / 2 ** (self.D - 1)

    # ----------------------------------------------------------------- rhs
    def rhs(self, w, ch=None, kappa=0.0):
        g = self.gamma
        glm = self.divb == "glm"
        ch2 = ch * ch if glm else None
        u = self.eval_points(w, self.Sv)
        R = np.zeros_like(w)
        for a in range(self.D):
            f = mhd.flux(u, a, g, ch2)
            R += np.einsum("cqv,q,rqv->cr", f, self.wv, self.Gv[a])
        R *= (2.0 / self.dxc)[:, None]
        if not glm:
            q = np.zeros((self.C, self.V))
            q[:, :8] = mhd.powell_q(self.means(w), g)
        for cL, cR, a, kind, sub in self.faces:
            SL = self.Ssub[(a, 1, sub)] if kind == 1 else self.Sf[(a, 1)]
            SR = self.Ssub[(a, -1, sub)] if kind == 2 else self.Sf[(a, -1)]
            wL = self.wf * (self.sub_w if kind == 1 else 1.0)
            wR = self.wf * (self.sub_w if kind == 2 else 1.0)
            uL = np.einsum("r,rpv->pv", w[cL], SL)
            uR = np.einsum("r,rpv->pv", w[cR], SR)
            interp = not glm and self.P.powell_q == "interp"
            if interp:
                F, BnF, qdL, qdR = self.face_state(uL[None], uR[None], a, ch, qdag=True)
                qdL, qdR = qdL[0], qdR[0]
            else:
                F, BnF = self.face_state(uL[None], uR[None], a, ch)
            F, BnF = F[0], BnF[0]
            mL, mR = 2.0 / self.dxc[cL], 2.0 / self.dxc[cR]
            R[cL] -= mL * np.einsum("pv,p,rpv->r", F, wL, SL)
            R[cR] += mR * np.einsum("pv,p,rpv->r", F, wR, SR)
            if not glm:
                jumpL = BnF - uL[:, mhd.BX + a]
                jumpR = -(BnF - uR[:, mhd.BX + a])
                if interp:   # q^dagger per face point and side, eq. powellq-interp
                    R[cL] -= mL * np.einsum("pv,rpv,p,p->r", qdL, SL, jumpL, wL)
                    R[cR] -= mR * np.einsum("pv,rpv,p,p->r", qdR, SR, jumpR, wR)
                else:
                    R[cL] -= mL * np.einsum("v,rpv,p,p->r", q[cL], SL, jumpL, wL)
                    R[cR] -= mR * np.einsum("v,rpv,p,p->r", q[cR], SR, jumpR, wR)
        out = R / self.mass
        if glm:
            psi_rows = [r for r, (k, v, i) in enumerate(self.rows) if k == "L" and v == mhd.PSI]
            out[:, psi_rows] -= kappa * w[:, psi_rows]
        return out

    # ------------------------------------------------------------------ dt
    def divb_face(self, w):
        acc = np.zeros(self.C)
        for cL, cR, a, kind, sub in self.faces:
            SL = self.Ssub[(a, 1, sub)] if kind == 1 else self.Sf[(a, 1)]
            SR = self.Ssub[(a, -1, sub)] if kind == 2 else self.Sf[(a, -1)]
            uL = np.einsum("r,rpv->pv", w[cL], SL)
            uR = np.einsum("r,rpv->pv", w[cR], SR)
            BnF = mhd.bn_face(uL[:, 0], uR[:, 0], uL[:, mhd.BX + a], uR[:, mhd.BX + a])
            # physical area of the face = fine face area
            dxf = min(self.dxc[cL], self.dxc[cR])
            area = (0.5 * dxf) ** (self.D - 1)
            acc[cL] += area * np.abs(BnF - uL[:, mhd.BX + a]) @ self.wf
            acc[cR] += area * np.abs(BnF - uR[:, mhd.BX + a]) @ self.wf
        return acc / self.dxc ** self.D

    def dt(self, w):
        g = self.gamma
        m = self.means(w)
        rho, v, p, Bv = mhd.primitives(m, g)
        c = mhd.signal_speed(m, g)
        s = np.sum(np.abs(v[:, : self.D]) + c[:, None], axis=1) / self.dxc
        dt = np.min(self.P.cfl / (2 * self.d + 1) / s)
        if self.divb == "powell":
            db = self.divb_face(w)
            rate = db * np.abs(np.sum(v * Bv, -1)) / m[:, mhd.EN]
            pos = rate > 0
            if np.any(pos):
                dt = min(dt, np.min(self.P.eta_powell / rate[pos]))
        return float(dt)

    def glm_speeds(self, dt):
        # AMR: a global, time-independent c_h (Sec. 4.1.5) must be given
        ch = self.P.c_h_fixed
        tau = max(self.P.c_r / ch, 3.0 * dt)
        return ch, 1.0 / tau

    # ---------------------------------------------------------------- helpers
    def project(self, fn, npts=None):
        npts = npts or self.d + 3
        qp, qw = B.gauss_tensor(self.D, npts)
        S = self.synth(qp)
        x = self.centers[:, None, :] + 0.5 * self.dxc[:, None, None] * qp[None, :, :]
        return np.einsum("cqv,q,rqv->cr", fn(x), qw, S) / self.mass

    def totals(self, w):
        return (self.means(w) * (self.dxc ** self.D)[:, None]).sum(0)

    def l1_error(self, w, fn_ref, npts=None):
        npts = npts or self.d + 3
        qp, qw = B.gauss_tensor(self.D, npts)
        u = self.eval_points(w, self.synth(qp))
        x = self.centers[:, None, :] + 0.5 * self.dxc[:, None, None] * qp[None, :, :]
        ur = fn_ref(x)
        cell = (0.5 * self.dxc) ** self.D / self.L ** self.D
        err = np.einsum("cqv,q,c->v", np.abs(u - ur), qw, cell)
        ref = np.einsum("cqv,q,c->v", np.abs(ur), qw, cell)
        return err, ref
