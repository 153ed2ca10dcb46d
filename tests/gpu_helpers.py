"""Shared helpers of the GPU tests: convert between the oracle's w[cell, row]
layout and the library's w[row][cell_stride] layout, and build nodal inputs."""
import numpy as np

from oracle import basis as OB


def to_device(w_oracle, solver, dtype=None):
    import torch
    C, N = w_oracle.shape
    assert N == solver.nrows and C == solver.ncell
    w = torch.zeros((solver.nrows, solver.stride), dtype=dtype or solver.dtype, device="cuda")
    w[:, :C] = torch.as_tensor(w_oracle.T.copy(), dtype=w.dtype, device="cuda")
    return w


def means_to_device(w_oracle, solver, scheme):
    """Degree-0 rows of the oracle state as the FP64 mean array of the FP32 form."""
    import torch
    rows = mean_rows(scheme)
    wm = torch.zeros((len(rows), solver.stride), dtype=torch.float64, device="cuda")
    wm[:, : solver.ncell] = torch.as_tensor(w_oracle[:, rows].T.copy(), device="cuda")
    return wm


def mean_rows(scheme):
    """Row indices of the degree-0 rows in the library's mean-row order."""
    n = scheme.n
    if scheme.divb == "glm":
        return [v * n for v in range(9)]
    ldf0 = 5 * n
    rows = [v * n for v in range(5)] + [ldf0 + j for j in range(scheme.D)]
    if scheme.D == 2:
        rows.append(ldf0 + len(scheme.ldf))
    return rows


def from_device(w, solver):
    return w[:, : solver.ncell].double().cpu().numpy().T.copy()


def nodal_input(scheme, fn, npts):
    """Conserved variables at the npts^D Gauss points of every cell, laid out
    [var][q][cell_stride] (points: tensor rule, last axis fastest)."""
    qp, _ = OB.gauss_tensor(scheme.D, npts)
    x = scheme.centers[:, None, :] + 0.5 * scheme.dx * qp[None, :, :]
    u = fn(x)  # [cell, q, var]
    return u


def nodal_to_device(u, solver):
    import torch
    C, Q, V = u.shape
    t = torch.zeros((V, Q, solver.stride), dtype=torch.float64, device="cuda")
    t[:, :, :C] = torch.as_tensor(np.transpose(u, (2, 1, 0)).copy(), device="cuda")
    return t


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
