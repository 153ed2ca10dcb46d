"""Plain FP64 CPU oracle of the DG-MHD spatial operator (test infrastructure).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this module. It is written from the paper, in the paper's order, with
numpy einsum / matmul as the only library primitives; it shares no code with
the CUDA library.

State layout used here: w[cell, row], rows = Legendre rows (var-major: var v,
mode l -> v*n + l) and, for the Powell scheme, one block of N_div LDF rows for
B (after the 5 hydro variables; in 2D B_z follows as a Legendre scalar).
Cells of a uniform periodic box are numbered x-fastest.

Passages followed:
* Sec. 3.1 eq. u-exp / x-xi: cell-local modal expansion on [-1,1]^D;
* Sec. 3.5 eq. wdot: M_l dw_l/dt = (2/dx)[ int f_a . d_a phi_l - oint F*.n phi_l ]
  + int s.phi_l  (the paper prints dx/2; the mapping xi = 2(x-x_c)/dx gives
  d/dx = (2/dx) d/dxi, which is what is used here);
* Sec. 3.5: Gauss-Legendre with d+1 points per dimension for volume and faces;
* Sec. 4.1.3 eq. powell-src-face with q^dagger = q(<u>_K) (eq. powellq-average,
  the default) or, with Params.powell_q = "interp", eq. powellq-interp against
  the HLLD interface state
  and B^n_F from eq. bxface-average-alfven;
* Sec. 4.1.5: GLM fluxes, upwinded psi*/B_n*, damping source -(c_h^2/c_p^2) psi,
  c_h = C'/(2d+1) dx/(D dt), c_r = c_p^2/c_h = 0.18, damping time >= 3 dt;
* Sec. 3.6 eq. cfl and Sec. 4.1.4 eq. powell_dt for the timestep;
* Sec. 3.6: SSP-RK3 (Shu-Osher form);
* Sec. 5.2.1 eq. lp_norm with d+3 points per dimension.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

from . import basis as B
from . import mhd


@dataclass
class Params:
    cfl: float = 0.3
    cfl_glm: float = 0.9      # C' of Sec. 4.1.5 (C < C' < 1)
    c_r: float = 0.18         # c_p^2 / c_h
    eta_powell: float = 0.2   # eq. powell_dt
    powell_q: str = "mean"    # q^dagger: "mean" eq. powellq-average (default), "interp" eq. powellq-interp
    eps_hlld: float = 1e-8
    Mtilde: float = 5.0       # Sec. 4.2.1 / 5.1
    beta: float = 2.0
    tvb_eps: float = 1e-8
    eps_rho: float = 1e-12
    eps_p: float = 1e-12
    rk_order: int = 3         # SSP-RK order 1..4 (Sec. 3.6); 0: d + 1, the paper's default


def ssp_rk_step(u, L, dt, order, lim=None):
    """One strong-stability-preserving Runge-Kutta step of order 1..4 for
    du/dt = L(u) (Sec. 3.6 uses SSP schemes of selectable order, see Gottlieb,
    Shu & Tadmor). u is the (already limited) step input; `lim` is applied to
    every later stage input before L evaluates it (Sec. 4.3).
    1: forward Euler.  2: SSPRK(2,2) and 3: SSPRK(3,3), Shu-Osher forms.
    4: Ketcheson's ten-stage SSPRK(10,4) in its low-storage form (Ketcheson
    2008): five forward-Euler stages of dt/6, a combination of the two
    registers, four more stages of dt/6 and a final stage of dt/10."""
    lim = lim or (lambda x: x)
    u0 = u
    if order == 1:
        return u0 + dt * L(u0)
    if order == 2:
        u1 = lim(u0 + dt * L(u0))
        return 0.5 * u0 + 0.5 * (u1 + dt * L(u1))
    if order == 3:
        u1 = lim(u0 + dt * L(u0))
        u2 = lim(0.75 * u0 + 0.25 * (u1 + dt * L(u1)))
        return u0 / 3.0 + 2.0 / 3.0 * (u2 + dt * L(u2))
    if order == 4:
        q1 = u0
        q2 = q1.copy()
        for i in range(5):
            if i:
                q1 = lim(q1)
            q1 = q1 + dt / 6.0 * L(q1)
        q2 = q2 / 25.0 + 9.0 / 25.0 * q1
        q1 = 15.0 * q2 - 5.0 * q1
        for _ in range(4):
            q1 = lim(q1)
            q1 = q1 + dt / 6.0 * L(q1)
        q1 = lim(q1)
        return q2 + 0.6 * q1 + dt / 10.0 * L(q1)
    raise ValueError(f"SSP-RK order {order} not in 1..4")


class Scheme:
    """DG-MHD on a uniform periodic box [0, L]^D with ncell cells per side."""

    def __init__(self, D: int, d: int, divb: str, gamma: float, ncell, L: float = 1.0,
                 params: Params | None = None):
        assert D in (2, 3) and divb in ("powell", "glm")
        self.D, self.d, self.divb, self.gamma = D, d, divb, gamma
        self.P = params or Params()
        self.ncell = tuple([ncell] * D) if np.isscalar(ncell) else tuple(ncell)
        self.L = L                      # side of the box along x; cells are cubes
        self.dx = L / self.ncell[0]
        self.C = int(np.prod(self.ncell))
        self.V = 9 if divb == "glm" else 8
        self.modes = B.mode_list(D, d)
        self.n = len(self.modes)
        self._build_rows()
        self._build_tables()
        self._build_mesh()

    # ------------------------------------------------------------------ basis
    def _build_rows(self):
        """rows: list of (kind, var or None, index). kind 'L' Legendre, 'B' LDF."""
        rows = []
        if self.divb == "glm":
            for v in range(9):
                rows += [("L", v, l) for l in range(self.n)]
        else:
            for v in range(5):
                rows += [("L", v, l) for l in range(self.n)]
            self.ldf = B.ldf_basis(self.D, self.d)
            rows += [("B", None, j) for j in range(len(self.ldf))]
            if self.D == 2:
                rows += [("L", mhd.BZ, l) for l in range(self.n)]
        self.rows = rows
        self.N = len(rows)
        self.legendre = [B.legendre_poly(k) for k in self.modes]
        mass = []
        for kind, v, i in rows:
            mass.append(B.legendre_mass(self.modes[i]) if kind == "L" else B.vdot(self.ldf[i], self.ldf[i]))
        self.mass_exact = mass
        self.mass = np.array([float(m) for m in mass])
        # mean rows: a Legendre row with mode 0; LDF rows of degree 0
        self.is_mean = np.array([(k == "L" and i == 0) or (k == "B" and B.pdegree(self.ldf[i][0]) <= 0
                                                            and all(B.pdegree(c) <= 0 for c in self.ldf[i]))
                                 for k, _, i in rows])

    def synth(self, pts, deriv=None):
        """S[r, q, v]: value (or d/dxi_deriv) of basis row r's component v at pts[q]."""
        S = np.zeros((self.N, len(pts), self.V))
        for r, (kind, v, i) in enumerate(self.rows):
            if kind == "L":
                poly = self.legendre[i] if deriv is None else B.pderiv(self.legendre[i], deriv)
                S[r, :, v] = B.peval(poly, pts)
            else:
                for a, comp in enumerate(self.ldf[i]):
                    poly = comp if deriv is None else B.pderiv(comp, deriv)
                    if poly:
                        S[r, :, mhd.BX + a] = B.peval(poly, pts)
        return S

    def face_points(self, axis, side, npts=None):
        """Points on the reference face xi_axis = side (tangential tensor Gauss,
        remaining axes in increasing order, last fastest) and their weights."""
        npts = npts or self.d + 1
        tp, tw = B.gauss_tensor(self.D - 1, npts) if self.D > 1 else (np.zeros((1, 0)), np.ones(1))
        pts = np.zeros((len(tw), self.D))
        others = [a for a in range(self.D) if a != axis]
        for j, a in enumerate(others):
            pts[:, a] = tp[:, j]
        pts[:, axis] = side
        return pts, tw

    def _build_tables(self):
        D = self.D
        self.qv, self.wv = B.gauss_tensor(D, self.d + 1)
        self.Sv = self.synth(self.qv)
        self.Gv = [self.synth(self.qv, deriv=a) for a in range(D)]
        self.Sf = {}
        for a in range(D):
            for s in (-1, 1):
                pts, wf = self.face_points(a, s)
                self.Sf[(a, s)] = self.synth(pts)
        self.wf = wf

    # ------------------------------------------------------------------- mesh
    def _build_mesh(self):
        idx = np.arange(self.C).reshape(self.ncell[::-1])  # [z][y][x] (x fastest)
        self.nbr_minus, self.nbr_plus = [], []
        for a in range(self.D):
            ax = self.D - 1 - a  # numpy axis of spatial axis a
            self.nbr_minus.append(np.roll(idx, 1, axis=ax).reshape(-1))
            self.nbr_plus.append(np.roll(idx, -1, axis=ax).reshape(-1))
        coords = np.stack(np.unravel_index(np.arange(self.C), self.ncell[::-1])[::-1], -1)
        self.centers = (coords + 0.5) * self.dx

    # -------------------------------------------------------------- evaluation
    def eval_points(self, w, S):
        return np.einsum("cr,rqv->cqv", w, S)

    def means(self, w):
        """Cell-mean conserved state <u>_K = 2^-D int u dxi (eq. powellq-average),
        by the volume Gauss rule (exact for the degree-d polynomials)."""
        u = self.eval_points(w, self.Sv)
        return np.einsum("cqv,q->cv", u, self.wv) / 2.0 ** self.D

    def project(self, fn, npts=None):
        """L2 projection (orthogonal basis, eq. basis-ortho) of fn(x[..., D]) ->
        conserved values [..., V], with npts (default d+3) Gauss points per dim."""
        npts = npts or self.d + 3
        qp, qw = B.gauss_tensor(self.D, npts)
        S = self.synth(qp)
        x = self.centers[:, None, :] + 0.5 * self.dx * qp[None, :, :]
        u = fn(x)
        return np.einsum("cqv,q,rqv->cr", u, qw, S) / self.mass

    # -------------------------------------------------------------------- rhs
    def glm_speeds(self, dt):
        """(c_h, damping rate c_h^2/c_p^2) for a uniform grid (Sec. 4.1.5)."""
        ch = self.P.cfl_glm / (2 * self.d + 1) * self.dx / (self.D * dt)
        tau = max(self.P.c_r / ch, 3.0 * dt)
        return ch, 1.0 / tau

    def face_state(self, uL, uR, axis, ch=None, qdag=False):
        """Numerical flux F* at face points and B^n_F (Sec. 4.1.2-4.1.5); with
        qdag also q^dagger of eq. powellq-interp for the left and the right
        trace against the HLLD interface state."""
        g = self.gamma
        rL, vL, pL, BL = mhd.primitives(uL, g)
        rR, vR, pR, BR = mhd.primitives(uR, g)
        BnL, BnR = BL[..., axis], BR[..., axis]
        BnF = mhd.bn_face(rL, rR, BnL, BnR)
        if qdag:
            F8, vF, BF = mhd.hlld(rL, vL, pL, BL, rR, vR, pR, BR, BnF, axis, g, self.P.eps_hlld, state=True)
            F = np.zeros(uL.shape)
            F[..., :8] = F8
            return F, BnF, mhd.powell_q_interp(vL, BL, vF, BF), mhd.powell_q_interp(vR, BR, vF, BF)
        F8 = mhd.hlld(rL, vL, pL, BL, rR, vR, pR, BR, BnF, axis, g, self.P.eps_hlld)
        F = np.zeros(uL.shape)
        F[..., :8] = F8
        if self.divb == "glm":
            bstar, pstar = mhd.glm_face(BnL, BnR, uL[..., mhd.PSI], uR[..., mhd.PSI], ch)
            F[..., mhd.BX + axis] = pstar
            F[..., mhd.PSI] = ch * ch * bstar
        return F, BnF

    def rhs(self, w, ch=None, kappa=0.0):
        """dw/dt of eq. wdot for every cell. GLM needs c_h and the damping rate."""
        g = self.gamma
        glm = self.divb == "glm"
        ch2 = ch * ch if glm else None
        u = self.eval_points(w, self.Sv)
        R = np.zeros_like(w)
        # volume integral  int f_a . d_a phi_l
        for a in range(self.D):
            f = mhd.flux(u, a, g, ch2)
            R += np.einsum("cqv,q,rqv->cr", f, self.wv, self.Gv[a])
        # surface integral  -oint F* . n phi_l  (and Powell's face term)
        if not glm:
            q = np.zeros((self.C, self.V))
            q[:, :8] = mhd.powell_q(self.means(w), g)
        for a in range(self.D):
            L = self.nbr_minus[a]
            uL = self.eval_points(w[L], self.Sf[(a, 1)])
            uR = self.eval_points(w, self.Sf[(a, -1)])
            interp = not glm and self.P.powell_q == "interp"
            if interp:
                F, BnF, qdL, qdR = self.face_state(uL, uR, a, ch, qdag=True)
            else:
                F, BnF = self.face_state(uL, uR, a, ch)
            contribL = np.einsum("cpv,p,rpv->cr", F, self.wf, self.Sf[(a, 1)])
            contribR = np.einsum("cpv,p,rpv->cr", F, self.wf, self.Sf[(a, -1)])
            R[L] -= contribL          # outward normal of L is +e_a
            R += contribR             # outward normal of R is -e_a
            if not glm:
                # -oint (q.phi_l)(B_F - B_K).n dS,  eq. powell-src-face
                jumpL = BnF - uL[..., mhd.BX + a]          # (B_F - B_L).(+e_a)
                jumpR = -(BnF - uR[..., mhd.BX + a])       # (B_F - B_R).(-e_a)
                if interp:   # q^dagger per face point and side, eq. powellq-interp
                    qphiL = np.einsum("cpv,rpv->cpr", qdL, self.Sf[(a, 1)])
                    qphiR = np.einsum("cpv,rpv->cpr", qdR, self.Sf[(a, -1)])
                else:
                    qphiL = np.einsum("cv,rpv->cpr", q[L], self.Sf[(a, 1)])
                    qphiR = np.einsum("cv,rpv->cpr", q, self.Sf[(a, -1)])
                R[L] -= np.einsum("cpr,cp,p->cr", qphiL, jumpL, self.wf)
                R -= np.einsum("cpr,cp,p->cr", qphiR, jumpR, self.wf)
        out = (2.0 / self.dx) * R / self.mass
        if glm:
            psi_rows = [r for r, (k, v, i) in enumerate(self.rows) if k == "L" and v == mhd.PSI]
            out[:, psi_rows] -= kappa * w[:, psi_rows]
        return out

    def rhs_local(self, wc, wnb, ch=None, kappa=0.0):
        """dw/dt of eq. wdot for a batch of cells given only their own weights
        wc[b, r] and their face neighbours' weights wnb[b, 2*axis + side, r]
        (side 0: the -axis neighbour, 1: the +axis neighbour). Same steps as
        `rhs`, for sampling a large box without holding all of it."""
        g = self.gamma
        glm = self.divb == "glm"
        ch2 = ch * ch if glm else None
        nb = len(wc)
        u = self.eval_points(wc, self.Sv)
        R = np.zeros_like(wc)
        for a in range(self.D):
            f = mhd.flux(u, a, g, ch2)
            R += np.einsum("cqv,q,rqv->cr", f, self.wv, self.Gv[a])
        if not glm:
            q = np.zeros((nb, self.V))
            q[:, :8] = mhd.powell_q(self.means(wc), g)
        for a in range(self.D):
            for side in (0, 1):
                wn = wnb[:, 2 * a + side]
                if side == 0:   # face with the -a neighbour: this cell is R
                    uL = self.eval_points(wn, self.Sf[(a, 1)])
                    uR = self.eval_points(wc, self.Sf[(a, -1)])
                    interp = not glm and self.P.powell_q == "interp"
                    if interp:
                        F, BnF, _, qd = self.face_state(uL, uR, a, ch, qdag=True)
                    else:
                        F, BnF = self.face_state(uL, uR, a, ch)
                    R += np.einsum("cpv,p,rpv->cr", F, self.wf, self.Sf[(a, -1)])
                    if not glm:
                        jump = -(BnF - uR[..., mhd.BX + a])
                        qphi = (np.einsum("cpv,rpv->cpr", qd, self.Sf[(a, -1)]) if interp
                                else np.einsum("cv,rpv->cpr", q, self.Sf[(a, -1)]))
                        R -= np.einsum("cpr,cp,p->cr", qphi, jump, self.wf)
                else:           # face with the +a neighbour: this cell is L
                    uL = self.eval_points(wc, self.Sf[(a, 1)])
                    uR = self.eval_points(wn, self.Sf[(a, -1)])
                    interp = not glm and self.P.powell_q == "interp"
                    if interp:
                        F, BnF, qd, _ = self.face_state(uL, uR, a, ch, qdag=True)
                    else:
                        F, BnF = self.face_state(uL, uR, a, ch)
                    R -= np.einsum("cpv,p,rpv->cr", F, self.wf, self.Sf[(a, 1)])
                    if not glm:
                        jump = BnF - uL[..., mhd.BX + a]
                        qphi = (np.einsum("cpv,rpv->cpr", qd, self.Sf[(a, 1)]) if interp
                                else np.einsum("cv,rpv->cpr", q, self.Sf[(a, 1)]))
                        R -= np.einsum("cpr,cp,p->cr", qphi, jump, self.wf)
        out = (2.0 / self.dx) * R / self.mass
        if glm:
            psi_rows = [r for r, (k, v, i) in enumerate(self.rows) if k == "L" and v == mhd.PSI]
            out[:, psi_rows] -= kappa * wc[:, psi_rows]
        return out

    # --------------------------------------------------------------------- dt
    def divb_face(self, w):
        """Face part of |div B|_K (App. C eq. divb-cell) in physical units:
        (1/V_K) oint |B^n_F - B^n_K| dS."""
        acc = np.zeros(self.C)
        for a in range(self.D):
            L = self.nbr_minus[a]
            uL = self.eval_points(w[L], self.Sf[(a, 1)])
            uR = self.eval_points(w, self.Sf[(a, -1)])
            rL = uL[..., mhd.RHO]
            rR = uR[..., mhd.RHO]
            BnF = mhd.bn_face(rL, rR, uL[..., mhd.BX + a], uR[..., mhd.BX + a])
            jl = np.abs(BnF - uL[..., mhd.BX + a]) @ self.wf
            jr = np.abs(BnF - uR[..., mhd.BX + a]) @ self.wf
            np.add.at(acc, L, jl)
            acc += jr
        # reference face measure -> physical: (dx/2)^(D-1); 1/V_K = dx^-D
        return acc * (0.5 * self.dx) ** (self.D - 1) / self.dx ** self.D

    def divb_norms(self, w):
        """Divergence diagnostics of App. C:
        cell:       |div B|_K, eq. divb-cell: (1/V_K) int_K |div B| (Gauss
                    points of the scheme) plus the face part (`divb_face`);
        total:      ||div B||_1 = (1/V) sum_K V_K |div B|_K, eq. divb-total;
        normalized: |div B|_K dx / |mean B|_K, eq. divb-normalized;
        signed:     (div B)_K = (1/V_K) oint B^n_F dS (outward normals),
                    eq. divb-gauss read with the cell volume V_K."""
        D, dx = self.D, self.dx
        div = sum(self.eval_points(w, self.Gv[a])[..., mhd.BX + a] for a in range(D)) * (2.0 / dx)
        vol = (np.abs(div) @ self.wv) / 2.0 ** D
        face = self.divb_face(w)
        sg = np.zeros(self.C)
        for a in range(D):
            L = self.nbr_minus[a]
            uL = self.eval_points(w[L], self.Sf[(a, 1)])
            uR = self.eval_points(w, self.Sf[(a, -1)])
            BnF = mhd.bn_face(uL[..., mhd.RHO], uR[..., mhd.RHO], uL[..., mhd.BX + a], uR[..., mhd.BX + a])
            flux = BnF @ self.wf
            np.add.at(sg, L, flux)      # +a face of the left cell
            sg -= flux                  # -a face of this cell
        sg *= (0.5 * dx) ** (D - 1) / dx ** D
        cell = vol + face
        Bm = mhd.primitives(self.means(w), self.gamma)[3]
        bmag = np.sqrt(np.sum(Bm * Bm, -1))
        return {"cell": cell, "volume": vol, "face": face, "signed": sg, "total": float(np.mean(cell)),
                "normalized": cell * dx / bmag}

    def dt(self, w):
        """Global dt: eq. cfl from cell means, and eq. powell_dt for Powell."""
        g = self.gamma
        m = self.means(w)
        rho, v, p, Bv = mhd.primitives(m, g)
        c = mhd.signal_speed(m, g)
        s = np.sum(np.abs(v[:, : self.D]) + c[:, None], axis=1) / self.dx
        dt = np.min(self.P.cfl / (2 * self.d + 1) / s)
        if self.divb == "powell":
            db = self.divb_face(w)
            rate = db * np.abs(np.sum(v * Bv, -1)) / m[:, mhd.EN]
            pos = rate > 0
            if np.any(pos):
                dt = min(dt, np.min(self.P.eta_powell / rate[pos]))
        return float(dt)

    # ------------------------------------------------------------------- step
    def rk_order(self):
        """SSP-RK order of a step: Params.rk_order, or d + 1 (at most 4) when 0."""
        return self.P.rk_order or min(self.d + 1, 4)

    def step(self, w, dt=None, limiter=None):
        """One SSP-RK step of order rk_order() (Sec. 3.6; `ssp_rk_step`).
        `limiter(w)` if given is applied to each stage input before it is
        evaluated (Sec. 4.3); dt (if not given) comes from the limited input."""
        lim = limiter or (lambda x: x)
        w0 = lim(w)
        dt = dt if dt is not None else self.dt(w0)
        ch, kappa = self.glm_speeds(dt) if self.divb == "glm" else (None, 0.0)
        return ssp_rk_step(w0, lambda x: self.rhs(x, ch, kappa), dt, self.rk_order(), lim), dt

    # ------------------------------------------------------------------ norms
    def l1_error(self, w, fn_ref, npts=None):
        """Per-variable L1 error, eq. lp_norm with d+3 points per dimension,
        together with the L1 norm of the reference."""
        npts = npts or self.d + 3
        qp, qw = B.gauss_tensor(self.D, npts)
        u = self.eval_points(w, self.synth(qp))
        x = self.centers[:, None, :] + 0.5 * self.dx * qp[None, :, :]
        ur = fn_ref(x)
        vol = float(np.prod(self.ncell)) * self.dx ** self.D
        cell = (0.5 * self.dx) ** self.D / vol
        err = np.einsum("cqv,q->v", np.abs(u - ur), qw) * cell
        ref = np.einsum("cqv,q->v", np.abs(ur), qw) * cell
        return err, ref

    def totals(self, w):
        """Volume integrals of the conserved variables (Sec. 4.1.3 conservation)."""
        m = self.means(w)
        return m.sum(0) * self.dx ** self.D
