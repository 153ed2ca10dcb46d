"""The closed-form workloads used by the convergence checks (Sec. 5.1.2
isodensity vortex, Sec. 5.2 3D Alfven wave) against properties the paper
states for them: periodicity, div B = 0, uniform density, constant |B|^2, and
the exact time dependence (advection by v0; a travelling wave at speed 2
along the cube diagonal). Central differences on a fine stencil."""
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
