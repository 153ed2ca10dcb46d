"""The closed-form workloads used by the convergence checks (Sec. 5.1.2
isodensity vortex, Sec. 5.2 3D Alfven wave) against properties the paper
states for them: periodicity, div B = 0, uniform density, constant |B|^2, and
the exact time dependence (advection by v0; a travelling wave at speed 2
along the cube diagonal). Central differences on a fine stencil. Also the
stated recipes of the seeded synthetic starts of the benchmark workloads
(decaying turbulence, smooth Fourier state)."""
import math

import numpy as np

from oracle import mhd
from paper_1806_02343_gb300 import workloads as W

G = 5.0 / 3.0


def _divergence(fn, x, h=1e-5):
    div = np.zeros(x.shape[:-1])
    for a in range(x.shape[-1]):
        e = np.zeros(x.shape[-1])
        e[a] = h
        div += (fn(x + e)[..., mhd.BX + a] - fn(x - e)[..., mhd.BX + a]) / (2 * h)
    return div


def test_alfven_3d_is_periodic_divergence_free_and_travels_at_speed_2():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (200, 3))
    u = W.alfven_3d(x)
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        assert np.abs(W.alfven_3d(x + e) - u).max() < 1e-11
    assert np.abs(_divergence(W.alfven_3d, x)).max() < 1e-8
    b2 = (u[:, mhd.BX:mhd.BZ + 1] ** 2).sum(-1)
    assert np.abs(b2 - b2[0]).max() < 1e-13                      # circular polarisation
    assert np.allclose(u[:, mhd.RHO], 1.0) and np.allclose(mhd.primitives(u, G)[2], 100.0)
    # u(x, t) = u(x - 2 t e1, 0)
    t = 0.137
    e1 = np.ones(3) / math.sqrt(3.0)
    assert np.abs(W.alfven_3d(x, t=t) - W.alfven_3d(x - 2 * t * e1)).max() < 1e-12


def test_isodensity_vortex_is_divergence_free_and_advected():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 20, (300, 2))
    u = W.isodensity_vortex_2d(x, alpha_deg=30.0)
    assert np.allclose(u[:, mhd.RHO], 1.0)
    assert np.abs(_divergence(lambda y: W.isodensity_vortex_2d(y, alpha_deg=30.0), x)).max() < 1e-8
    a = math.radians(30.0)
    v0 = math.sqrt(2.0) * np.array([math.cos(a), math.sin(a)])
    t = 3.3
    assert np.abs(W.isodensity_vortex_2d(x, t=t, alpha_deg=30.0)
                  - W.isodensity_vortex_2d(x - v0 * t, alpha_deg=30.0)).max() < 1e-12
    # far from the centre the state is the background: rho = 1, p = 1, v = v0, B = 0
    far = W.isodensity_vortex_2d(np.array([[0.5, 0.5]]), alpha_deg=30.0)[0]
    rho, v, p, B = mhd.primitives(far[None], G)
    assert abs(p[0] - 1.0) < 1e-12 and np.abs(v[0, :2] - v0).max() < 1e-12 and np.abs(B).max() < 1e-12


def test_turbulence_recipe():
    """The decaying-turbulence start of the 256^3 workload: random-phase
    solenoidal velocity (every Fourier amplitude perpendicular to its k), power
    only on 2 <= |k| <= 8 with shell energy falling as k^-2, rms Mach 2 at
    c_s = sqrt(5/3) on a grid other than the one that set the scale, periodic;
    rho = 1, p = 1, B = (0.5, 0, 0), psi = 0; the grid and pointwise paths agree."""
    T = W.Turbulence3D(nvar=9)
    K = T.KMAX
    ks = np.arange(-K, K + 1)
    kx, ky, kz = np.meshgrid(ks, ks, ks, indexing="ij")
    kv = np.stack([kx, ky, kz], -1).astype(float)
    kk = np.linalg.norm(kv, axis=-1)
    assert np.abs(np.einsum("abcd,abcd->abc", T.A, kv)).max() < 1e-12           # k . A_k = 0
    power = np.sum(np.abs(T.A) ** 2, -1)
    assert power[(kk < 2) | (kk > 8)].max() == 0.0
    shells = np.arange(2, 9)
    E = np.array([power[(kk >= s - 0.5) & (kk < s + 0.5)].sum() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(E), 1)[0]
    assert abs(slope + 2.0) < 0.3
    g = (np.arange(37) + 0.31) / 37                                             # not the 48^3 scaling grid
    v = T.grid_velocity(g, g, g)
    mach = math.sqrt(float(np.mean(np.sum(v * v, -1)))) / math.sqrt(G)
    assert abs(mach - 2.0) < 0.02
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (50, 3))
    u = T(x)
    assert np.abs(T(x + np.array([1.0, 0.0, 0.0])) - u).max() < 1e-10
    rho, vel, p, Bv = mhd.primitives(u[:, :8], G)
    assert np.allclose(rho, 1.0) and np.allclose(p, 1.0) and np.allclose(Bv, [0.5, 0.0, 0.0])
    assert np.all(u[:, 8] == 0.0)
    # the separable grid evaluation equals the pointwise one
    gx, gy, gz = np.array([0.1, 0.6]), np.array([0.25]), np.array([0.9, 0.05, 0.5])
    grid = T.grid_velocity(gx, gy, gz)
    pts = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), -1)
    assert np.abs(T.state_from_velocity(grid) - T(pts)).max() < 1e-11


def test_smooth_fourier_recipe():
    """The seeded smooth Fourier state of the 64^3 degree-3 workload: 8 modes
    per component with integer 1 <= |k| <= 4, amplitudes in (0, 1); rho within
    1 +- 0.2 and of mean 1; |v_i| <= 0.3; p = 1; B = curl A divergence-free,
    periodic, max |B_i| = 0.3 on the 64^3 scaling grid."""
    F = W.SmoothFourier3D(nvar=9)
    for k, a, ph in [F.rho_m] + list(F.v_m) + list(F.A_m):
        nk = np.linalg.norm(k, axis=1)
        assert k.shape == (8, 3) and np.all(k == np.round(k)) and np.all((nk >= 1) & (nk <= 4))
        assert np.all((a > 0) & (a < 1)) and len(set(map(tuple, k))) == 8
    g = (np.arange(64) + 0.5) / 64
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)
    u = F(X)
    rho, v, p, Bv = mhd.primitives(u[..., :8], G)
    assert np.abs(rho - 1.0).max() <= 0.2 + 1e-12 and abs(rho.mean() - 1.0) < 1e-12
    assert np.abs(v).max() <= 0.3 + 1e-12 and np.allclose(p, 1.0)
    assert abs(np.abs(Bv).max() - 0.3) < 1e-12
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (100, 3))
    assert np.abs(F(x + np.array([0.0, 1.0, 0.0])) - F(x)).max() < 1e-12
    assert np.abs(_divergence(F, x)).max() < 1e-7
