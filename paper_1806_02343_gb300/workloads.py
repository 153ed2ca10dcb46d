"""Seeded synthetic initial conditions shared by the tests, the oracle side and
the benchmark.

This module holds no DG arithmetic: it only defines the analytic fields of the
workloads (functions of physical position returning conserved variables) and
the seeded random mode tables they use. Both the CUDA path and the CPU oracle
project these fields with their own code.

Variables: (rho, m_x, m_y, m_z, E, B_x, B_y, B_z[, psi]); positions x[..., D]
in the periodic unit box. Functions work on numpy arrays and, where noted, on
torch tensors (any device) so that large inputs can be built on the GPU.
"""
from __future__ import annotations

import math
import numpy as np


def _xp(x):
    if isinstance(x, np.ndarray):
        return np
    import torch
    return torch


def _assemble(xp, rho, vx, vy, vz, p, bx, by, bz, gamma, nvar):
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    comps = [rho, rho * vx, rho * vy, rho * vz, E, bx, by, bz]
    if nvar == 9:
        comps.append(xp.zeros_like(rho))
    return xp.stack(comps, -1)


# ---------------------------------------------------------------------------
# 2D circularly polarised Alfven wave (Sec. 5.2.3), scaled to the unit box
# ---------------------------------------------------------------------------

ALFVEN2D_K = (2, 1)      # wave vector 2*pi*(2, 1): periodic in the unit box


def alfven_2d(x, t=0.0, gamma=5.0 / 3.0, eps=0.1, nvar=8):
    """Exact solution at time t. The wave propagates along e_par = k/|k|
    (angle atan(1/2) = 26.57 deg to x) at v_A = B_par/sqrt(rho) = 1 towards
    negative x_par; rho = 1, p = 0.1, B_par = 1, amplitude eps."""
    xp = _xp(x)
    kx, ky = ALFVEN2D_K
    kn = math.hypot(kx, ky)
    ca, sa = kx / kn, ky / kn
    # phase 2*pi*k.x shifted by the travelled distance t along e_par (v_A = 1)
    xpar = x[..., 0] * ca + x[..., 1] * sa + t
    phi = 2.0 * math.pi * kn * xpar
    one = xp.ones_like(phi)
    bperp = eps * xp.sin(phi)
    bz = eps * xp.cos(phi)
    bx = ca * one - sa * bperp
    by = sa * one + ca * bperp
    vx = -sa * bperp
    vy = ca * bperp
    vz = bz
    return _assemble(xp, one, vx, vy, vz, 0.1 * one, bx, by, bz, gamma, nvar)


def isodensity_vortex_2d(x, t=0.0, alpha_deg=45.0, gamma=5.0 / 3.0, eta=1.0, xi=1.0, L=20.0, nvar=8):
    """Isodensity MHD vortex (Sec. 5.1.2), exact solution at time t on the
    periodic box [0, L)^2 (the paper's [-10, 10]^2 shifted by L/2): rho = 1, the
    background p = 1 and v0 = sqrt(2) (cos a, sin a); with psi = exp((1-r^2)/2),
    dv = eta/(2 pi) curl(0, 0, psi), dB = xi/(2 pi) curl(0, 0, psi),
    dp = [xi^2 (1 - r^2) - eta^2] exp(1 - r^2) / (8 pi^2); advected: u(x - v0 t, 0)."""
    xp = _xp(x)
    a = math.radians(alpha_deg)
    v0x, v0y = math.sqrt(2.0) * math.cos(a), math.sqrt(2.0) * math.sin(a)
    X = xp.remainder(x[..., 0] - v0x * t, L) - 0.5 * L
    Y = xp.remainder(x[..., 1] - v0y * t, L) - 0.5 * L
    r2 = X * X + Y * Y
    psi = xp.exp(0.5 * (1.0 - r2))
    one = xp.ones_like(r2)
    # curl(0, 0, psi) = (d_y psi, -d_x psi, 0) = psi (-Y, X, 0)
    cv, cb = eta / (2.0 * math.pi), xi / (2.0 * math.pi)
    p = 1.0 + (xi * xi * (1.0 - r2) - eta * eta) * xp.exp(1.0 - r2) / (8.0 * math.pi ** 2)
    return _assemble(xp, one, v0x - cv * psi * Y, v0y + cv * psi * X, 0.0 * one, p,
                     -cb * psi * Y, cb * psi * X, 0.0 * one, gamma, nvar)


def alfven_3d(x, t=0.0, gamma=5.0 / 3.0, eps=0.02, nvar=8):
    """Circularly polarised Alfven wave in 3D (Sec. 5.2), exact solution at time
    t on the periodic unit cube: rho = 1, p = 100; in the frame e1 = (1,1,1)/sqrt(3),
    e2 = (1,-1,0)/sqrt(2), e3 = e1 x e2, v = e1 + eps (cos phi e2 + sin phi e3),
    B = e1 - eps (cos phi e2 + sin phi e3), phi = 2 pi / lambda (x.e1 - 2t) with
    lambda = 1/sqrt(3) (periodic along every axis; Alfven speed 1 plus the flow
    speed 1 along e1)."""
    xp = _xp(x)
    s3, s2, s6 = math.sqrt(3.0), math.sqrt(2.0), math.sqrt(6.0)
    e1 = (1 / s3, 1 / s3, 1 / s3)
    e2 = (1 / s2, -1 / s2, 0.0)
    e3 = (1 / s6, 1 / s6, -2 / s6)
    xpar = (x[..., 0] + x[..., 1] + x[..., 2]) / s3
    phi = 2.0 * math.pi * s3 * (xpar - 2.0 * t)
    c, sn = eps * xp.cos(phi), eps * xp.sin(phi)
    one = xp.ones_like(phi)
    v = [e1[k] * one + c * e2[k] + sn * e3[k] for k in range(3)]
    Bf = [e1[k] * one - c * e2[k] - sn * e3[k] for k in range(3)]
    return _assemble(xp, one, v[0], v[1], v[2], 100.0 * one, Bf[0], Bf[1], Bf[2], gamma, nvar)


# ---------------------------------------------------------------------------
# entropy (density) wave: uniform v, p, B; advected density (pin case)
# ---------------------------------------------------------------------------


def entropy_wave(x, t=0.0, D=3, gamma=5.0 / 3.0, v0=(1.0, 0.5, 0.25), B0=(0.3, -0.2, 0.1), amp=0.2,
                 k=(1, 0, 0), nvar=8):
    xp = _xp(x)
    ph = 0.0
    for a in range(D):
        ph = ph + k[a] * (x[..., a] - v0[a] * t)
    rho = 1.0 + amp * xp.sin(2.0 * math.pi * ph)
    one = xp.ones_like(rho)
    return _assemble(xp, rho, v0[0] * one, v0[1] * one, v0[2] * one, one, B0[0] * one, B0[1] * one,
                     B0[2] * one, gamma, nvar)


def uniform_state(x, gamma=5.0 / 3.0, nvar=8, rho=1.3, v=(0.4, -0.7, 0.2), p=0.8, B=(0.6, 0.3, -0.5)):
    xp = _xp(x)
    one = xp.ones_like(x[..., 0])
    return _assemble(xp, rho * one, v[0] * one, v[1] * one, v[2] * one, p * one, B[0] * one, B[1] * one,
                     B[2] * one, gamma, nvar)


# ---------------------------------------------------------------------------
# smooth seeded Fourier state (3D, 64^3 degree-3 GLM workload)
# ---------------------------------------------------------------------------


def fourier_modes(seed=1234, nmodes=8, kmax=4, ncomp=1):
    """nmodes integer wave vectors with 1 <= |k| <= kmax, amplitudes U(0,1),
    phases U(0, 2pi), per component."""
    rng = np.random.default_rng(seed)
    cand = [k for k in np.ndindex(2 * kmax + 1, 2 * kmax + 1, 2 * kmax + 1)]
    cand = np.array(cand) - kmax
    nrm = np.linalg.norm(cand, axis=1)
    cand = cand[(nrm >= 1) & (nrm <= kmax)]
    out = []
    for _ in range(ncomp):
        idx = rng.choice(len(cand), size=nmodes, replace=False)
        out.append((cand[idx].astype(np.float64), rng.uniform(0, 1, nmodes), rng.uniform(0, 2 * np.pi, nmodes)))
    return out


def _fsum(xp, x, k, a, ph):
    s = 0.0
    for j in range(len(a)):
        s = s + a[j] * xp.cos(2.0 * math.pi * (k[j, 0] * x[..., 0] + k[j, 1] * x[..., 1] + k[j, 2] * x[..., 2])
                              + ph[j])
    return s / np.sum(a)


def _fsum_curl(xp, x, modes):
    """curl of A, A_i = sum_j a_j cos(2 pi k_j.x + ph_j) / sum a (analytic)."""
    dA = []  # dA[i][a] = d A_i / d x_a
    for (k, a, ph) in modes:
        der = []
        for ax in range(3):
            s = 0.0
            for j in range(len(a)):
                s = s - a[j] * 2.0 * math.pi * k[j, ax] * xp.sin(
                    2.0 * math.pi * (k[j, 0] * x[..., 0] + k[j, 1] * x[..., 1] + k[j, 2] * x[..., 2]) + ph[j])
            der.append(s / np.sum(a))
        dA.append(der)
    return (dA[2][1] - dA[1][2], dA[0][2] - dA[2][0], dA[1][0] - dA[0][1])


class SmoothFourier3D:
    """rho = 1 + 0.2 sum_j a_j cos(2 pi k_j.x + ph_j)/sum a_j (8 modes, |k| <= 4);
    v_i built the same way with amplitude 0.3; B = curl A (A built the same
    way) rescaled so max |B_i| = 0.3 on a 64^3 sample grid; p = 1."""

    def __init__(self, seed=1234, gamma=5.0 / 3.0, nvar=9):
        m = fourier_modes(seed, ncomp=7)
        self.rho_m, self.v_m, self.A_m = m[0], m[1:4], m[4:7]
        self.gamma, self.nvar = gamma, nvar
        g = (np.arange(64) + 0.5) / 64
        X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)
        bx, by, bz = _fsum_curl(np, X, self.A_m)
        self.bscale = 0.3 / max(np.abs(bx).max(), np.abs(by).max(), np.abs(bz).max())

    def __call__(self, x):
        xp = _xp(x)
        rho = 1.0 + 0.2 * _fsum(xp, x, *self.rho_m)
        v = [0.3 * _fsum(xp, x, *m) for m in self.v_m]
        b = [self.bscale * c for c in _fsum_curl(xp, x, self.A_m)]
        return _assemble(xp, rho, v[0], v[1], v[2], xp.ones_like(rho), b[0], b[1], b[2], self.gamma, self.nvar)


# ---------------------------------------------------------------------------
# 3D Orszag-Tang extrusion and MHD blast
# ---------------------------------------------------------------------------


def orszag_tang_3d(x, gamma=5.0 / 3.0, nvar=8):
    xp = _xp(x)
    tp = 2.0 * math.pi
    X, Y = x[..., 0], x[..., 1]
    one = xp.ones_like(X)
    rho = 25.0 / (36.0 * math.pi) * one
    p = 5.0 / (12.0 * math.pi) * one
    s = 1.0 / math.sqrt(4.0 * math.pi)
    return _assemble(xp, rho, -xp.sin(tp * Y), xp.sin(tp * X), 0.0 * one, p, -s * xp.sin(tp * Y),
                     s * xp.sin(2.0 * tp * X), 0.0 * one, gamma, nvar)


def blast_3d(x, gamma=5.0 / 3.0, nvar=8, center=(0.5, 0.5, 0.5), r0=0.1, p_in=100.0, p_out=0.1,
             B0=(10.0 / math.sqrt(4.0 * math.pi), 0.0, 0.0)):
    """MHD blast: p = p_in inside r < r0, p_out outside, rho = 1, v = 0, uniform B0."""
    xp = _xp(x)
    r2 = (x[..., 0] - center[0]) ** 2 + (x[..., 1] - center[1]) ** 2 + (x[..., 2] - center[2]) ** 2
    one = xp.ones_like(r2)
    p = p_out * one + (p_in - p_out) * (r2 < r0 * r0)
    zero = 0.0 * one
    return _assemble(xp, one, zero, zero, zero, p, B0[0] * one, B0[1] * one, B0[2] * one, gamma, nvar)


def blast_params(seed):
    """Seeded blast variant for indicator training: centre in [0.3, 0.7]^3,
    radius 0.05-0.15, pressure ratio 10^2-10^4 (outside p = 0.1), field of
    strength 0-10/sqrt(4 pi) along a random direction."""
    rng = np.random.default_rng(seed)
    center = tuple(rng.uniform(0.3, 0.7, 3))
    r0 = rng.uniform(0.05, 0.15)
    ratio = 10.0 ** rng.uniform(2.0, 4.0)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    bmag = rng.uniform(0.0, 10.0 / math.sqrt(4.0 * math.pi))
    return dict(center=center, r0=r0, p_in=0.1 * ratio, p_out=0.1, B0=tuple(bmag * d))


# ---------------------------------------------------------------------------
# decaying-turbulence start (3D, 256^3 degree-2 GLM workload)
# ---------------------------------------------------------------------------


class Turbulence3D:
    """Random-phase solenoidal velocity with E(k) ~ k^-2 on 2 <= |k| <= 8,
    rescaled to rms Mach 2 (c_s = sqrt(gamma p / rho) = sqrt(5/3)); uniform
    B0 = (0.5, 0, 0), rho = 1, p = 1; seed 1234.

    v(x) = Re sum_k A_k exp(2 pi i k.x), A_k perpendicular to k. Evaluation is
    separable over axes so a whole grid of points can be built with three small
    contractions (see `grid_velocity`)."""

    KMAX = 8

    def __init__(self, seed=1234, gamma=5.0 / 3.0, nvar=9, mach=2.0):
        rng = np.random.default_rng(seed)
        K = self.KMAX
        ks = np.arange(-K, K + 1)
        kx, ky, kz = np.meshgrid(ks, ks, ks, indexing="ij")
        kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        sel = (kk >= 2) & (kk <= 8)
        amp = np.zeros(kk.shape)
        # shell energy E(k) ~ k^-2 spread over ~4 pi k^2 modes: |A|^2 ~ k^-4
        amp[sel] = kk[sel] ** -2.0
        A = np.zeros(kk.shape + (3,), dtype=np.complex128)
        r = rng.normal(size=kk.shape + (3,)) + 1j * rng.normal(size=kk.shape + (3,))
        kv = np.stack([kx, ky, kz], -1).astype(np.float64)
        knorm = np.where(kk > 0, kk, 1.0)[..., None]
        khat = kv / knorm
        r = r - np.sum(r * khat, -1, keepdims=True) * khat          # solenoidal
        rn = np.linalg.norm(r, axis=-1, keepdims=True)
        r = r / np.where(rn > 0, rn, 1.0)
        A = r * amp[..., None]
        A[~sel] = 0.0
        self.A = A
        self.gamma, self.nvar = gamma, nvar
        cs = math.sqrt(gamma * 1.0 / 1.0)
        # rms of Re sum: 0.5 * sum |A_k|^2 (modes are distinct and non-conjugate
        # in general; pair k, -k adds cross terms, measured on a sample below)
        g = (np.arange(48) + 0.5) / 48
        v = self._eval_np(g, g, g)
        rms = math.sqrt(float(np.mean(np.sum(v * v, -1))))
        self.scale = mach * cs / rms

    def _eval_np(self, gx, gy, gz):
        K = self.KMAX
        ks = np.arange(-K, K + 1)
        ex = np.exp(2j * np.pi * np.outer(ks, gx))
        ey = np.exp(2j * np.pi * np.outer(ks, gy))
        ez = np.exp(2j * np.pi * np.outer(ks, gz))
        out = []
        for c in range(3):
            t = np.einsum("abc,ck->abk", self.A[..., c], ez)
            t = np.einsum("abk,bj->ajk", t, ey)
            t = np.einsum("ajk,ai->ijk", t, ex)
            out.append(t.real)
        return np.stack(out, -1)

    def grid_velocity(self, gx, gy, gz):
        """Velocity on the tensor grid gx x gy x gz (arrays of coordinates;
        numpy or torch), shape [nx, ny, nz, 3], already scaled to Mach 2."""
        if isinstance(gx, np.ndarray):
            return self.scale * self._eval_np(gx, gy, gz)
        import torch
        dev = gx.device
        K = self.KMAX
        ks = torch.arange(-K, K + 1, device=dev, dtype=torch.float64)
        ex = torch.exp(2j * math.pi * torch.outer(ks, gx.double()).to(torch.complex128))
        ey = torch.exp(2j * math.pi * torch.outer(ks, gy.double()).to(torch.complex128))
        ez = torch.exp(2j * math.pi * torch.outer(ks, gz.double()).to(torch.complex128))
        out = []
        for c in range(3):
            Ac = torch.as_tensor(self.A[..., c], device=dev)
            t = torch.einsum("abc,ck->abk", Ac, ez)
            t = torch.einsum("abk,bj->ajk", t, ey)
            t = torch.einsum("ajk,ai->ijk", t, ex)
            out.append(t.real)
        return self.scale * torch.stack(out, -1)

    def state_from_velocity(self, v):
        xp = _xp(v)
        one = xp.ones_like(v[..., 0])
        return _assemble(xp, one, v[..., 0], v[..., 1], v[..., 2], one, 0.5 * one, 0.0 * one, 0.0 * one,
                         self.gamma, self.nvar)

    def __call__(self, x):
        """Pointwise evaluation (numpy; small inputs): x[..., 3]."""
        K = self.KMAX
        ks = np.arange(-K, K + 1)
        ph = np.exp(2j * np.pi * np.einsum("...a,k->...ak", x, ks))  # [..., 3, nk]
        v = np.einsum("abcd,...a,...b,...c->...d", self.A, ph[..., 0, :], ph[..., 1, :], ph[..., 2, :]).real
        return self.state_from_velocity(self.scale * v)


# ---------------------------------------------------------------------------
# point values at the Gauss points of every cell of a uniform box (input
# layout of dg_mhd_project: [var][q][cell], cell x-fastest, q last-axis-fastest)
# ---------------------------------------------------------------------------


def gauss_nodal(fn, n, npts, D=3, stride=None, device="cuda"):
    """Evaluates fn (torch-capable) at the npts^D Gauss-Legendre points of each
    cell of an n^D periodic unit box; returns a float64 tensor [V][Q][stride]."""
    import torch
    g1, _ = np.polynomial.legendre.leggauss(npts)
    c1 = ((torch.arange(n, device=device, dtype=torch.float64)[:, None] + 0.5
           + 0.5 * torch.as_tensor(g1, device=device)[None, :]) / n).reshape(-1)
    if D == 3:
        X, Y, Z = torch.meshgrid(c1, c1, c1, indexing="ij")
        U = fn(torch.stack([X, Y, Z], -1))
        V = U.shape[-1]
        U = U.reshape(n, npts, n, npts, n, npts, V).permute(6, 1, 3, 5, 4, 2, 0).reshape(V, npts ** 3, n ** 3)
    else:
        X, Y = torch.meshgrid(c1, c1, indexing="ij")
        U = fn(torch.stack([X, Y], -1))
        V = U.shape[-1]
        U = U.reshape(n, npts, n, npts, V).permute(4, 1, 3, 2, 0).reshape(V, npts ** 2, n ** 2)
    stride = stride or U.shape[-1]
    out = torch.zeros((V, U.shape[1], stride), dtype=torch.float64, device=device)
    out[:, :, : U.shape[-1]] = U
    return out


# ---------------------------------------------------------------------------
# static octree meshes (input description: leaves, refinement and 2:1 balance)
# ---------------------------------------------------------------------------


def octree_leaves(D, base_level, max_level, refine):
    """Leaves [(level, (i, j[, k]))] of a periodic unit box: start uniform at
    base_level, split every leaf for which refine(center, dx, level) is true
    (level by level up to max_level), then split coarse leaves until every face
    neighbour of a leaf is at most one level coarser (2:1 balance).
    Returned in Morton (Z-curve) order of the leaf's lower corner."""
    leaves = set()
    n0 = 2 ** base_level
    for k in np.ndindex(*([n0] * D)):
        leaves.add((base_level, tuple(int(x) for x in k)))
    for lvl in range(base_level, max_level):
        new = set()
        for (l, k) in leaves:
            if l == lvl:
                dx = 1.0 / 2 ** l
                ctr = np.array([(x + 0.5) * dx for x in k])
                if refine(ctr, dx, l):
                    for ch in np.ndindex(*([2] * D)):
                        new.add((l + 1, tuple(2 * x + int(c) for x, c in zip(k, ch))))
                    continue
            new.add((l, k))
        leaves = new

    def cover(l, k):
        for j in range(l + 1):
            key = (l - j, tuple(x >> j for x in k))
            if key in leaves:
                return key
        return None

    changed = True
    while changed:
        changed = False
        for (l, k) in list(leaves):
            if (l, k) not in leaves:
                continue
            n = 2 ** l
            for a in range(D):
                for s in (-1, 1):
                    kk = list(k)
                    kk[a] = (kk[a] + s) % n
                    cv = cover(l, tuple(kk))
                    if cv is not None and cv[0] < l - 1:
                        cl, ck = cv
                        leaves.discard(cv)
                        for ch in np.ndindex(*([2] * D)):
                            leaves.add((cl + 1, tuple(2 * x + int(c) for x, c in zip(ck, ch))))
                        changed = True

    def morton(item):
        l, k = item
        sh = max_level - l
        key = 0
        coords = [x << sh for x in k]
        for bit in range(max_level, -1, -1):
            for a in range(D - 1, -1, -1):
                key = (key << 1) | ((coords[a] >> bit) & 1)
        return (key, l)

    return sorted(leaves, key=morton)


def turbulence_nodal(n, npts, stride, device="cuda", seed=1234, nvar=9, mach=2.0):
    """Decaying-turbulence start at the npts^3 Gauss points of every cell of an
    n^3 box, laid out [var][q][stride] (built slab by slab on the device)."""
    import torch
    g1, _ = np.polynomial.legendre.leggauss(npts)
    T = Turbulence3D(seed=seed, nvar=nvar, mach=mach)
    coords = ((torch.arange(n, device=device, dtype=torch.float64)[:, None] + 0.5
               + 0.5 * torch.as_tensor(g1, device=device)[None, :]) / n).reshape(-1)
    Q = npts ** 3
    nodal = torch.zeros((nvar, Q, stride), dtype=torch.float64, device=device)
    zs = max(1, 2 ** 22 // (n * n))
    for z0 in range(0, n, zs):
        z1 = min(n, z0 + zs)
        v = T.grid_velocity(coords, coords, coords[z0 * npts:z1 * npts])
        U = T.state_from_velocity(v)
        nz = z1 - z0
        U = U.reshape(n, npts, n, npts, nz, npts, nvar).permute(6, 1, 3, 5, 4, 2, 0).reshape(nvar, Q, nz * n * n)
        nodal[:, :, z0 * n * n:z1 * n * n] = U
        del v, U
    return nodal


def morton_order(levels, ijk, D, max_level):
    """Permutation sorting leaves by the Z-curve key of their lower corner."""
    lv = np.asarray(levels, dtype=np.int64)
    k = np.asarray(ijk, dtype=np.int64).reshape(len(lv), D) << (max_level - lv)[:, None]
    key = np.zeros(len(lv), dtype=np.uint64)
    for bit in range(max_level, -1, -1):
        for a in range(D - 1, -1, -1):
            key = (key << np.uint64(1)) | ((k[:, a] >> bit) & 1).astype(np.uint64)
    return np.lexsort((lv, key))


def orszag_tang_octree(lo=4, hi=7, target=1_500_000, tol=0.1):
    """Static octree for the 3D Orszag-Tang extrusion: a 2:1-balanced quadtree
    in (x, y) refined where dx * max|grad B| of the initial field exceeds a
    threshold (the density is uniform at t = 0, so B drives the refinement),
    extruded along z (cubic cells: a leaf of level l spans 2^l cells in z).
    The threshold is bisected to reach about `target` leaves.
    Returns (levels int8 [N], ijk int32 [N, 3]) in Morton order."""
    s = 1.0 / math.sqrt(4.0 * math.pi)

    def grad(c):
        return max(2 * math.pi * s * abs(math.cos(2 * math.pi * c[1])),
                   4 * math.pi * s * abs(math.cos(4 * math.pi * c[0])))

    def build(theta):
        q = octree_leaves(2, lo, hi, lambda c, dx, l: dx * grad(c) > theta)
        return q, sum(2 ** l for l, _ in q)

    a, b = 0.0, 10.0
    q, n = build(0.5 * (a + b))
    for _ in range(30):
        th = 0.5 * (a + b)
        q, n = build(th)
        if abs(n - target) <= tol * target:
            break
        if n > target:
            a = th
        else:
            b = th
    lev, ijk = [], []
    for l, (i, j) in q:
        nz = 2 ** l
        lev.append(np.full(nz, l, dtype=np.int8))
        ijk.append(np.stack([np.full(nz, i), np.full(nz, j), np.arange(nz)], 1))
    lev = np.concatenate(lev)
    ijk = np.concatenate(ijk).astype(np.int32)
    perm = morton_order(lev, ijk, 3, hi)
    return lev[perm], ijk[perm]


def leaf_nodal(fn, levels, ijk, npts, stride, D=3, device="cuda"):
    """fn at the npts^D Gauss points of every leaf (unit box), laid out
    [var][q][stride] (q: last axis fastest)."""
    import torch
    g1, _ = np.polynomial.legendre.leggauss(npts)
    qp = np.stack(np.meshgrid(*([g1] * D), indexing="ij"), -1).reshape(-1, D)
    lv = torch.as_tensor(np.asarray(levels, dtype=np.float64), device=device)
    dx = torch.pow(2.0, -lv)
    k = torch.as_tensor(np.asarray(ijk, dtype=np.float64).reshape(len(levels), D), device=device)
    ctr = (k + 0.5) * dx[:, None]
    N = len(levels)
    out = None
    chunk = 1 << 20
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        x = ctr[c0:c1, None, :] + 0.5 * dx[c0:c1, None, None] * torch.as_tensor(qp, device=device)[None]
        U = fn(x)                                   # [cells, Q, V]
        if out is None:
            out = torch.zeros((U.shape[-1], qp.shape[0], stride), dtype=torch.float64, device=device)
        out[:, :, c0:c1] = U.permute(2, 1, 0)
    return out
