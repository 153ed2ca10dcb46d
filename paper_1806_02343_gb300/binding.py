"""ctypes binding of the C ABI in include/dg_mhd.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module only loads it,
passes device pointers from torch tensors and the current CUDA stream, and
turns status codes into exceptions. There is no CPU fallback: if the library
is missing, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdgmhd.so")

DG_OK, DG_W_FLOOR = 0, 1
DG_E_TIMEOUT = -6
DG_DIVB_POWELL, DG_DIVB_GLM = 0, 1
DG_PREC_FP64, DG_PREC_FP32MIX = 0, 1
DG_LIMIT_OFF, DG_LIMIT_TVB, DG_LIMIT_MLP = 0, 1, 2

# every entry point declared in include/dg_mhd.h
EXPORTS = [
    "dg_mhd_default_params", "dg_mhd_init", "dg_mhd_state_layout", "dg_mhd_project", "dg_mhd_set_glm",
    "dg_mhd_rhs", "dg_mhd_limit", "dg_mhd_dt", "dg_mhd_step", "dg_mhd_last_dt", "dg_mhd_status",
    "dg_mhd_profile", "dg_mhd_profile_read", "dg_mhd_launch_count", "dg_mhd_rhs_noalloc", "dg_mhd_destroy",
    "dg_mhd_strerror", "dg_mhd_mlp_features", "dg_mhd_mlp_set_weights", "dg_mhd_mlp_infer", "dg_mhd_mlp_loss_grad",
    "dg_mhd_mlp_train", "dg_mhd_counters", "dg_mhd_positivity_listed", "dg_mhd_ldf_legendre", "dg_mhd_limiter_counts", "dg_mhd_divb", "dg_mhd_smoothness",
    "dg_mhd_amr_marks", "dg_mhd_regrid_plan", "dg_mhd_remap", "dg_mhd_regrid_plan_mesh",
    "dg_mhd_sibling_groups", "dg_mhd_octree_faces", "dg_mhd_basis_values", "dg_mhd_regrid_tables",
    "dg_mhd_probe", "dg_mhd_stage", "dg_mhd_set_dt", "dg_mhd_set_owned", "dg_mhd_glm_speeds",
]
KIND_FACE, KIND_CELL, KIND_DT, KIND_LIMIT, KIND_PROJECT, KIND_POSITIVITY, KIND_MLP = range(7)


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int32 * 3), ("box_len", ctypes.c_double),
                ("periodic", ctypes.c_int), ("n_leaves", ctypes.c_int64),
                ("level", ctypes.POINTER(ctypes.c_int8)), ("ijk", ctypes.POINTER(ctypes.c_int32)),
                ("partial", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("cfl", "cfl_glm", "c_r", "c_h_fixed", "eta_powell", "eps_hlld",
                                               "Mtilde", "beta", "tvb_eps", "eps_rho", "eps_p")] + \
               [(k, ctypes.c_int) for k in ("precision", "limiter", "positivity", "generic_kernels", "rk_order",
                                            "powell_q")]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p
    L.dg_mhd_default_params.argtypes = [ctypes.POINTER(Params)]
    L.dg_mhd_default_params.restype = None
    L.dg_mhd_init.argtypes = [ctypes.POINTER(MeshDesc), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.dg_mhd_state_layout.argtypes = [vp, i64p, i64p, i64p, i64p]
    L.dg_mhd_project.argtypes = [vp, dp, ctypes.c_int, vp, dp, vp]
    L.dg_mhd_set_glm.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp]
    L.dg_mhd_rhs.argtypes = [vp, vp, dp, vp, dp, vp]
    L.dg_mhd_limit.argtypes = [vp, vp, dp, vp, vp]
    L.dg_mhd_stage.argtypes = [vp, vp, dp, vp, dp, vp, dp, ctypes.c_double, ctypes.c_double, vp]
    L.dg_mhd_set_dt.argtypes = [vp, dp, vp]
    L.dg_mhd_set_owned.argtypes = [vp, vp, vp]
    L.dg_mhd_glm_speeds.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.dg_mhd_dt.argtypes = [vp, vp, dp, dp, vp]
    L.dg_mhd_step.argtypes = [vp, vp, dp, dp, vp]
    L.dg_mhd_last_dt.argtypes = [vp]
    L.dg_mhd_last_dt.restype = ctypes.c_void_p
    L.dg_mhd_status.argtypes = [vp, ctypes.c_int]
    L.dg_mhd_profile.argtypes = [vp, ctypes.c_int]
    L.dg_mhd_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), i64p]
    L.dg_mhd_launch_count.argtypes = [vp]
    L.dg_mhd_launch_count.restype = ctypes.c_int64
    L.dg_mhd_rhs_noalloc.argtypes = [ctypes.POINTER(MeshDesc), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(Params), ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
    L.dg_mhd_mlp_features.argtypes = [vp, vp, dp, vp, ctypes.c_int, vp]
    L.dg_mhd_mlp_set_weights.argtypes = [vp, vp, ctypes.c_int, ctypes.c_float]
    L.dg_mhd_mlp_infer.argtypes = [vp, vp, dp, vp, vp, vp]
    L.dg_mhd_mlp_loss_grad.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int, vp, ctypes.c_float, vp,
                                       vp, vp]
    L.dg_mhd_mlp_train.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int, vp, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_double), vp]
    L.dg_mhd_positivity_listed.argtypes = [vp, i64p, ctypes.c_int]
    L.dg_mhd_ldf_legendre.argtypes = [ctypes.c_int, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
    L.dg_mhd_counters.argtypes = [vp, i64p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_int]
    L.dg_mhd_limiter_counts.argtypes = [vp, i64p, i64p, i64p, ctypes.c_int]
    L.dg_mhd_divb.argtypes = [vp, vp, vp, vp, vp, vp]
    L.dg_mhd_limiter_counts.restype = ctypes.c_int
    L.dg_mhd_smoothness.argtypes = [vp, vp, dp, ctypes.c_int, vp, vp]
    L.dg_mhd_amr_marks.argtypes = [vp, vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    L.dg_mhd_regrid_plan.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, i64p]
    L.dg_mhd_remap.argtypes = [vp, vp, vp, vp, dp, vp, dp, vp]
    L.dg_mhd_regrid_plan_mesh.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, vp, i64p]
    L.dg_mhd_sibling_groups.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, i64p]
    L.dg_mhd_octree_faces.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp, vp,
                                      i64p]
    ip = ctypes.POINTER(ctypes.c_int)
    L.dg_mhd_regrid_tables.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp]
    L.dg_mhd_basis_values.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, ctypes.c_int64, vp,
                                      ip, ip]
    L.dg_mhd_probe.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), vp]
    L.dg_mhd_destroy.argtypes = [vp]
    L.dg_mhd_destroy.restype = None
    L.dg_mhd_strerror.argtypes = [ctypes.c_int]
    L.dg_mhd_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if not hasattr(L, name):
            raise RuntimeError(f"{LIB_PATH} does not export {name}")
    _lib = L
    return L


class DGError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {lib().dg_mhd_strerror(code).decode()} ({code})")
        self.code = code


def _check(code, what):
    if code < 0:
        raise DGError(code, what)
    return code


def wait(stream=None, timeout_s=60.0, poll_s=1e-4, event=None):
    """Host-side watchdog on stream completion: records an event on the stream
    (default: the current one) and polls it until the work before it has
    finished, raising DGError(DG_E_TIMEOUT) once timeout_s has passed instead
    of blocking inside the driver. The device work is not cancelled; the
    caller decides what to do with a stream that did not finish. `event`:
    an already recorded object with a query() method (tests inject one)."""
    import time
    if event is None:
        import torch
        event = torch.cuda.Event()
        event.record(stream if stream is not None else torch.cuda.current_stream())
    deadline = time.monotonic() + timeout_s
    while not event.query():
        if time.monotonic() > deadline:
            raise DGError(DG_E_TIMEOUT, f"stream not complete after {timeout_s:g} s")
        time.sleep(poll_s)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def mesh_desc(dim, n, box_len=1.0) -> MeshDesc:
    m = MeshDesc()
    m.n_leaves = 0
    m.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for a in range(3):
        m.n[a] = nn[a]
    m.box_len = box_len
    m.periodic = 1
    return m


def rhs_noalloc(dim, n, degree, divb, w, out, gamma=5.0 / 3.0, box_len=1.0, c_h=0.0, damping_rate=0.0,
                status=None):
    """dg_mhd_rhs_noalloc: the operator with all device scratch in the library's
    static array (for callers that must not allocate device memory). w and out:
    contiguous CUDA float64 tensors of shape (state rows, cells rounded up to 32);
    status: optional CUDA int32 tensor of one element that receives the call's
    device status word."""
    import torch
    dim_n = [int(x) for x in (n if isinstance(n, (tuple, list)) else (n,) * dim)]
    ncell = 1
    for x in dim_n[:dim]:
        ncell *= x
    stride = (ncell + 31) // 32 * 32
    nv = ctypes.c_int()
    nr = ctypes.c_int()
    scheme = DG_DIVB_GLM if divb == "glm" else DG_DIVB_POWELL
    _check(lib().dg_mhd_basis_values(dim, degree, scheme, 0, None, 0, None, ctypes.byref(nr), ctypes.byref(nv)),
           "dg_mhd_basis_values")
    for name, t in (("w", w), ("out", out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and tuple(t.shape) == (nr.value, stride)):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape ({nr.value}, {stride})")
    if status is not None and not (isinstance(status, torch.Tensor) and status.is_cuda
                                   and status.dtype == torch.int32 and status.numel() >= 1):
        raise ValueError("status must be a CUDA int32 tensor with at least one element")
    m = mesh_desc(dim, n, box_len)
    _check(lib().dg_mhd_rhs_noalloc(ctypes.byref(m), degree, scheme, gamma, None, c_h, damping_rate, _ptr(w),
                                    _ptr(out), _ptr(status) if status is not None else None, _stream()),
           "dg_mhd_rhs_noalloc")


PROBE_FP32_FMA, PROBE_FP64_FMA, PROBE_TF32_MMA, PROBE_COPY = range(4)


def probe(kind, nbytes=1 << 30):
    """dg_mhd_probe: (rate, ms) of one timed launch on the current device; rate in
    flop/s (FMA and MMA kinds) or bytes/s read plus written (copy: two device
    buffers of nbytes are allocated here)."""
    import torch
    rate, ms = ctypes.c_double(), ctypes.c_double()
    src = dst = None
    if kind == PROBE_COPY:
        src = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
        dst = torch.empty_like(src)
    _check(lib().dg_mhd_probe(kind, _ptr(src), _ptr(dst), nbytes if kind == PROBE_COPY else 0, ctypes.byref(rate),
                              ctypes.byref(ms), _stream()), "dg_mhd_probe")
    return rate.value, ms.value


def _leaf_arrays(levels, ijk):
    import numpy as np
    lev = np.ascontiguousarray(levels, dtype=np.int8)
    k = np.ascontiguousarray(ijk, dtype=np.int32)
    if k.ndim != 2 or k.shape[0] != lev.shape[0]:
        raise ValueError("ijk must be [n, dim] with one row per level")
    return lev, k


def sibling_groups(levels, ijk):
    """Groups of 2^dim sibling leaves of an octree mesh (host, no GPU):
    int32 [n_groups, 2^dim], the leaf index of each octant."""
    import numpy as np
    lev, k = _leaf_arrays(levels, ijk)
    dim, n, ng = k.shape[1], lev.shape[0], ctypes.c_int64()
    _check(lib().dg_mhd_sibling_groups(dim, n, lev.ctypes.data, k.ctypes.data, 0, None, ctypes.byref(ng)),
           "dg_mhd_sibling_groups")
    out = np.zeros((ng.value, 1 << dim), dtype=np.int32)
    _check(lib().dg_mhd_sibling_groups(dim, n, lev.ctypes.data, k.ctypes.data, ng.value, out.ctypes.data,
                                       ctypes.byref(ng)), "dg_mhd_sibling_groups")
    return out


def basis_values(dim, degree, divb, xi):
    """The basis at reference points xi [P, dim] in [-1, 1]^dim (host, no GPU):
    float64 [rows, vars, P]; u_v(xi_p) = sum_r out[r, v, p] w[r]."""
    import numpy as np
    x = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, dim)
    scheme = DG_DIVB_GLM if divb == "glm" else DG_DIVB_POWELL
    R, V = ctypes.c_int(), ctypes.c_int()
    P = x.shape[0]
    _check(lib().dg_mhd_basis_values(dim, degree, scheme, P, x.ctypes.data, 0, None, ctypes.byref(R),
                                     ctypes.byref(V)), "dg_mhd_basis_values")
    out = np.zeros((R.value, V.value, P), dtype=np.float64)
    _check(lib().dg_mhd_basis_values(dim, degree, scheme, P, x.ctypes.data, out.size, out.ctypes.data,
                                     ctypes.byref(R), ctypes.byref(V)), "dg_mhd_basis_values")
    return out


def ldf_legendre(degree):
    """The 3D LDF -> componentwise Legendre map of the specialised Powell
    kernels (host, no GPU): float64 [n_div, 3, n_modes] with
    B_c = sum_j w_j sum_l A[j, c, l] P_l."""
    import numpy as np
    nd, nm = ctypes.c_int(), ctypes.c_int()
    _check(lib().dg_mhd_ldf_legendre(degree, 0, None, ctypes.byref(nd), ctypes.byref(nm)), "dg_mhd_ldf_legendre")
    out = np.zeros((nd.value, 3, nm.value), dtype=np.float64)
    _check(lib().dg_mhd_ldf_legendre(degree, out.size, out.ctypes.data, ctypes.byref(nd), ctypes.byref(nm)),
           "dg_mhd_ldf_legendre")
    return out


def cell_points(dim, npts, box_len=1.0, n=None, levels=None, ijk=None, device="cpu"):
    """Physical coordinates of the npts^dim Gauss-Legendre points of every cell
    in the order dg_mhd_project takes them (cells in mesh order; points with
    the last axis fastest): float64 [cells, npts^dim, dim]. Uniform box: n
    cells per axis of size box_len / n[0], numbered x-fastest; octree: levels
    and ijk [cells, dim] in a cube of side box_len."""
    import numpy as np
    import torch
    g, _ = np.polynomial.legendre.leggauss(npts)
    g = torch.as_tensor(g, dtype=torch.float64, device=device)
    grids = torch.meshgrid(*([g] * dim), indexing="ij")
    qp = torch.stack([x.reshape(-1) for x in grids], -1)           # [Q, dim]
    if levels is None:
        nn = [int(x) for x in list(n)[:dim]]
        r = torch.arange(int(np.prod(nn)), device=device)
        ks = []
        for a in range(dim):
            ks.append(r % nn[a])
            r = r // nn[a]
        k = torch.stack(ks, -1).to(torch.float64)
        size = torch.full((k.shape[0], 1), box_len / nn[0], dtype=torch.float64, device=device)
    else:
        lev = torch.as_tensor(np.asarray(levels, dtype=np.float64), device=device)
        size = (box_len / torch.pow(2.0, lev))[:, None]
        k = torch.as_tensor(np.asarray(ijk, dtype=np.float64).reshape(-1, dim), device=device)
    centers = (k + 0.5) * size
    return centers[:, None, :] + 0.5 * size[:, None, :] * qp[None, :, :]


def mean_rows(dim, degree, divb, nrows):
    """State rows of the degree-0 fields, in the order of the FP64 mean array:
    Legendre mode 0 of each variable, then the degree-0 LDF rows, row order."""
    n = math.comb(degree + dim, dim)
    if divb == "glm":
        return [v * n for v in range(9)]
    rows = [v * n for v in range(5)] + [5 * n + j for j in range(dim)]
    if dim == 2:
        rows.append(nrows - n)                     # B_z mode 0 after the LDF rows
    return rows


def eval_points(table, w, mean=None, wmean=None):
    """Point values [vars, P, cells] (float64) from the basis table of
    basis_values [rows, vars, P] and state rows w [rows, cells] (any device);
    with wmean [len(mean), cells] the FP64 means replace the float mean rows."""
    import torch
    W = w.to(torch.float64)
    if wmean is not None:
        W = W.clone()
        W[mean] = wmean.to(torch.float64)
    T = torch.as_tensor(table, dtype=torch.float64, device=W.device)
    return torch.einsum("rvp,rc->vpc", T, W)


def regrid_tables(dim, degree, divb):
    """The regridding tables of a context (host, no GPU): dict of float64
    arrays QL [dim, n, n], QB [dim, dim, nd, nd], PL / RL [2^dim, n, n],
    PB / RB [2^dim, nd, nd] (nd = 0 for GLM)."""
    import numpy as np
    scheme = DG_DIVB_GLM if divb == "glm" else DG_DIVB_POWELL
    sizes = np.zeros(6, dtype=np.int64)
    _check(lib().dg_mhd_regrid_tables(dim, degree, scheme, 0, None, sizes.ctypes.data), "dg_mhd_regrid_tables")
    flat = np.zeros(int(sizes.sum()), dtype=np.float64)
    _check(lib().dg_mhd_regrid_tables(dim, degree, scheme, flat.size, flat.ctypes.data, sizes.ctypes.data),
           "dg_mhd_regrid_tables")
    n, no = math.comb(degree + dim, dim), 1 << dim
    nd = int(round(math.sqrt(sizes[3] / no))) if sizes[3] else 0
    shapes = {"QL": (dim, n, n), "QB": (dim, dim, nd, nd), "PL": (no, n, n), "PB": (no, nd, nd),
              "RL": (no, n, n), "RB": (no, nd, nd)}
    out, o = {}, 0
    for key, size in zip(("QL", "QB", "PL", "PB", "RL", "RB"), sizes):
        out[key] = flat[o:o + size].reshape(shapes[key])
        o += size
    return out


def octree_faces(levels, ijk, partial=False):
    """Faces of an octree mesh as a context builds them (host, no GPU): int32
    arrays left cell, right cell, meta (axis | kind << 2 | sub << 4). partial:
    a partition's local mesh (faces with no leaf across them left out)."""
    import numpy as np
    lev, k = _leaf_arrays(levels, ijk)
    dim, n, nf = k.shape[1], lev.shape[0], ctypes.c_int64()
    pf = 1 if partial else 0
    _check(lib().dg_mhd_octree_faces(dim, n, lev.ctypes.data, k.ctypes.data, pf, 0, None, None, None,
                                     ctypes.byref(nf)), "dg_mhd_octree_faces")
    out = [np.zeros(nf.value, dtype=np.int32) for _ in range(3)]
    _check(lib().dg_mhd_octree_faces(dim, n, lev.ctypes.data, k.ctypes.data, pf, nf.value,
                                     *(o.ctypes.data for o in out), ctypes.byref(nf)), "dg_mhd_octree_faces")
    return tuple(out)


def regrid_plan_mesh(levels, ijk, marks):
    """New leaves (levels int8, ijk int32 [n, dim]) and their sources (int32
    [n, 2]) from per-leaf marks, without a context (host, no GPU)."""
    import numpy as np
    lev, k = _leaf_arrays(levels, ijk)
    mk = np.ascontiguousarray(marks, dtype=np.int8)
    if mk.shape != lev.shape:
        raise ValueError("one mark per leaf")
    dim, n, nn = k.shape[1], lev.shape[0], ctypes.c_int64()
    _check(lib().dg_mhd_regrid_plan_mesh(dim, n, lev.ctypes.data, k.ctypes.data, mk.ctypes.data, 0, None, None,
                                         None, ctypes.byref(nn)), "dg_mhd_regrid_plan_mesh")
    lev_n = np.zeros(nn.value, dtype=np.int8)
    ijk_n = np.zeros((nn.value, dim), dtype=np.int32)
    src = np.zeros((nn.value, 2), dtype=np.int32)
    _check(lib().dg_mhd_regrid_plan_mesh(dim, n, lev.ctypes.data, k.ctypes.data, mk.ctypes.data, nn.value,
                                         lev_n.ctypes.data, ijk_n.ctypes.data, src.ctypes.data, ctypes.byref(nn)),
           "dg_mhd_regrid_plan_mesh")
    return lev_n, ijk_n, src


def mlp_loss_grad(X, y, theta, nin, pos_weight=1.0):
    """Loss and gradient of the indicator network on the device (FP32)."""
    import torch
    grad = torch.zeros_like(theta)
    loss = torch.zeros(1, dtype=torch.float64, device=theta.device)
    _check(lib().dg_mhd_mlp_loss_grad(_ptr(X), X.shape[1], _ptr(y), X.shape[0], nin, _ptr(theta), pos_weight,
                                      _ptr(grad), _ptr(loss), _stream()), "dg_mhd_mlp_loss_grad")
    return float(loss.item()), grad


def mlp_train(X, y, theta, nin, epochs, batch, lr=1e-3, pos_weight=1.0, seed=0):
    last = ctypes.c_double()
    _check(lib().dg_mhd_mlp_train(_ptr(X), X.shape[1], _ptr(y), X.shape[0], nin, _ptr(theta), epochs, batch, lr,
                                  pos_weight, seed, ctypes.byref(last), _stream()), "dg_mhd_mlp_train")
    return last.value


def default_params(**kw) -> Params:
    p = Params()
    lib().dg_mhd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Solver:
    """Owns one dg_mhd_ctx. State tensors are allocated by the caller (torch) with
    the layout reported by dg_mhd_state_layout: w[row][cell_stride]."""

    def __init__(self, dim, n, degree, divb, gamma=5.0 / 3.0, box_len=1.0, leaves=None, levels=None, ijk=None,
                 partial=False, **params):
        """n: cells per axis of a uniform box, or None with `leaves` =
        [(level, (i, j[, k]))] for an octree mesh of a cube of side box_len."""
        import numpy as np
        import torch
        L = lib()
        m = MeshDesc()
        m.dim = dim
        nn = (list(n) if n is not None else [1, 1, 1]) + [1] * (3 - len(n or []))
        for a in range(3):
            m.n[a] = nn[a]
        m.box_len = box_len
        m.periodic = 1
        if leaves is not None:
            levels = [l for l, _ in leaves]
            ijk = [k for _, k in leaves]
        self._n, self._lev, self._ijk = (nn[:dim] if levels is None else None), None, None
        if levels is not None:
            self._lev = np.ascontiguousarray(np.asarray(levels, dtype=np.int8))
            self._ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1))
            m.n_leaves = len(self._lev)
            m.level = self._lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
            m.ijk = self._ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            m.partial = 1 if partial else 0
        self.params = default_params(**params)
        self.divb = divb
        h = ctypes.c_void_p()
        _check(L.dg_mhd_init(ctypes.byref(m), degree, DG_DIVB_GLM if divb == "glm" else DG_DIVB_POWELL, gamma,
                             ctypes.byref(self.params), ctypes.byref(h)), "dg_mhd_init")
        self.h = h
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        _check(L.dg_mhd_state_layout(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
               "dg_mhd_state_layout")
        self.nrows, self.nmean, self.ncell, self.stride = a.value, b.value, c.value, d.value
        self.fp32 = self.params.precision == DG_PREC_FP32MIX
        self.dtype = torch.float32 if self.fp32 else torch.float64
        self.dim, self.degree = dim, degree
        self.gamma, self.box_len = gamma, box_len

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().dg_mhd_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # ------------------------------------------------------------- point values
    def project_ic(self, fn, w, wmean=None, npts=None):
        """L2 projection of fn onto the basis (dg_mhd_project): fn takes the
        cells' Gauss points x [cells, points, dim] (float64 on w's device) and
        returns the conserved variables [cells, points, vars]; npts points per
        axis (default degree + 3, at most 8). Holds [vars][points][stride]
        doubles at once: for very large meshes fill dg_mhd_project's input in
        slabs instead."""
        import torch
        npts = npts or min(8, self.degree + 3)
        x = cell_points(self.dim, npts, self.box_len, self._n, self._lev, self._ijk, w.device)
        u = fn(x)
        nodal = torch.zeros((u.shape[-1], x.shape[1], self.stride), dtype=torch.float64, device=w.device)
        nodal[:, :, : self.ncell] = torch.as_tensor(u, dtype=torch.float64, device=w.device).permute(2, 1, 0)
        self.project(nodal, npts, w, wmean)

    def mean_rows(self):
        return mean_rows(self.dim, self.degree, self.divb, self.nrows)

    def eval_at_points(self, w, wmean=None, xi=None):
        """Conserved variables at reference points xi [P, dim] in [-1, 1]^dim
        of every cell: float64 [vars, P, ncell] on w's device (the FP64 means
        used where given), independent of the basis ordering."""
        table = basis_values(self.dim, self.degree, self.divb, xi)
        wm = None if wmean is None else wmean[:, : self.ncell]
        return eval_points(table, w[:, : self.ncell], self.mean_rows(), wm)

    # ------------------------------------------------------------- buffers
    def alloc_state(self, device="cuda"):
        import torch
        w = torch.zeros((self.nrows, self.stride), dtype=self.dtype, device=device)
        wm = torch.zeros((self.nmean, self.stride), dtype=torch.float64, device=device) if self.fp32 else None
        return w, wm

    # ------------------------------------------------------------- entry points
    def project(self, nodal, npts, w, wmean=None):
        _check(lib().dg_mhd_project(self.h, _ptr(nodal), npts, _ptr(w), _ptr(wmean), _stream()), "dg_mhd_project")

    def set_glm(self, ch, kappa):
        _check(lib().dg_mhd_set_glm(self.h, ch, kappa, _stream()), "dg_mhd_set_glm")

    def rhs(self, w, wmean, out, outmean=None):
        _check(lib().dg_mhd_rhs(self.h, _ptr(w), _ptr(wmean), _ptr(out), _ptr(outmean), _stream()), "dg_mhd_rhs")

    def limit(self, w, wmean=None, troubled=None):
        return _check(lib().dg_mhd_limit(self.h, _ptr(w), _ptr(wmean), _ptr(troubled), _stream()),
                      "dg_mhd_limit")

    def dt(self, w, wmean=None, out=None):
        import torch
        if out is None:
            out = torch.zeros(1, dtype=torch.float64, device=w.device)
        _check(lib().dg_mhd_dt(self.h, _ptr(w), _ptr(wmean), _ptr(out), _stream()), "dg_mhd_dt")
        return out

    def stage(self, w, wmean, u0, u0mean, out, outmean, a, b):
        """out = a u0 + b (w + dt L(w)) with the context's current dt (dg_mhd_stage)."""
        _check(lib().dg_mhd_stage(self.h, _ptr(w), _ptr(wmean), _ptr(u0), _ptr(u0mean), _ptr(out), _ptr(outmean),
                                  a, b, _stream()), "dg_mhd_stage")

    def set_dt(self, dt):
        """dt (and the GLM speeds) from a one-element CUDA float64 tensor."""
        _check(lib().dg_mhd_set_dt(self.h, _ptr(dt), _stream()), "dg_mhd_set_dt")

    def glm_speeds(self):
        """(c_h, damping rate) of the context (host floats; synchronises)."""
        ch, kap = ctypes.c_double(), ctypes.c_double()
        _check(lib().dg_mhd_glm_speeds(self.h, ctypes.byref(ch), ctypes.byref(kap)), "dg_mhd_glm_speeds")
        return ch.value, kap.value

    def set_owned(self, mask):
        """Cells that count in the timestep minimum (CUDA uint8 tensor of n_cells), or None."""
        _check(lib().dg_mhd_set_owned(self.h, _ptr(mask), _stream()), "dg_mhd_set_owned")

    def step(self, w, wmean=None, dt=None):
        _check(lib().dg_mhd_step(self.h, _ptr(w), _ptr(wmean), _ptr(dt), _stream()), "dg_mhd_step")

    def last_dt_ptr(self):
        return lib().dg_mhd_last_dt(self.h)

    def profile(self, enable):
        _check(lib().dg_mhd_profile(self.h, 1 if enable else 0), "dg_mhd_profile")

    def profile_read(self, kind):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().dg_mhd_profile_read(self.h, kind, ctypes.byref(ms), ctypes.byref(n)), "dg_mhd_profile_read")
        return ms.value, n.value

    def launch_count(self):
        return lib().dg_mhd_launch_count(self.h)

    # --------------------------------------------------------- learned indicator
    def n_features(self):
        return 8 * {2: {0: 1, 1: 3, 2: 6, 3: 10}, 3: {0: 1, 1: 4, 2: 10, 3: 20}}[self.dim][self.degree] + 10 * self.dim

    def mlp_features(self, w, wmean, X, ldx):
        _check(lib().dg_mhd_mlp_features(self.h, _ptr(w), _ptr(wmean), _ptr(X), ldx, _stream()),
               "dg_mhd_mlp_features")

    def mlp_set_weights(self, theta, threshold=0.5):
        _check(lib().dg_mhd_mlp_set_weights(self.h, _ptr(theta), self.n_features(), threshold),
               "dg_mhd_mlp_set_weights")

    def mlp_infer(self, w, wmean=None, flags=None, prob=None):
        _check(lib().dg_mhd_mlp_infer(self.h, _ptr(w), _ptr(wmean), _ptr(flags), _ptr(prob), _stream()),
               "dg_mhd_mlp_infer")

    def counters(self, reset=False):
        n, m, e = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(lib().dg_mhd_counters(self.h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e), 1 if reset else 0),
               "dg_mhd_counters")
        return {"pos_cells": n.value, "inj_mass": m.value, "inj_energy": e.value}

    def positivity_listed(self, reset=False):
        """Cells the FP32 positivity screen sent to the full procedure, summed
        over limiter passes since the last reset (dg_mhd_positivity_listed)."""
        n = ctypes.c_int64()
        _check(lib().dg_mhd_positivity_listed(self.h, ctypes.byref(n), 1 if reset else 0), "dg_mhd_positivity_listed")
        return n.value

    # ------------------------------------------------------------ regridding
    def smoothness(self, w, wmean=None, fields=(0, 5, 6, 7)):
        """Smoothness indicator (Sec. 5): per cell the max over the monitored
        conserved components `fields` and the directions (FP64 device tensor)."""
        import torch
        s = torch.zeros(self.stride, dtype=torch.float64, device=w.device)
        mask = sum(1 << f for f in fields)
        _check(lib().dg_mhd_smoothness(self.h, _ptr(w), _ptr(wmean), mask, _ptr(s), _stream()), "dg_mhd_smoothness")
        return s[: self.ncell]

    def amr_marks(self, w, wmean=None, fields=(0, 5, 6, 7), s_tilde=0.03, min_level=0, max_level=17):
        """Refinement marks (+1 refine, -1 coarsen with the sibling group, 0) and
        the smoothness indicator, as device tensors."""
        import torch
        marks = torch.zeros(self.stride, dtype=torch.int8, device=w.device)
        s = torch.zeros(self.stride, dtype=torch.float64, device=w.device)
        mask = sum(1 << f for f in fields)
        _check(lib().dg_mhd_amr_marks(self.h, _ptr(w), _ptr(wmean), mask, s_tilde, min_level, max_level,
                                      _ptr(marks), _ptr(s), _stream()), "dg_mhd_amr_marks")
        return marks[: self.ncell], s[: self.ncell]

    def regrid_plan(self, marks):
        """New leaves (levels int8, ijk int32 [n, dim]) and their sources
        (int32 [n, 2]) from host or device marks."""
        import numpy as np
        mk = np.ascontiguousarray(marks.cpu().numpy() if hasattr(marks, "cpu") else np.asarray(marks), dtype=np.int8)
        n = ctypes.c_int64()
        _check(lib().dg_mhd_regrid_plan(self.h, mk.ctypes.data, 0, None, None, None, ctypes.byref(n)),
               "dg_mhd_regrid_plan")
        lev = np.zeros(n.value, dtype=np.int8)
        ijk = np.zeros((n.value, self.dim), dtype=np.int32)
        src = np.zeros((n.value, 2), dtype=np.int32)
        _check(lib().dg_mhd_regrid_plan(self.h, mk.ctypes.data, n.value, lev.ctypes.data, ijk.ctypes.data,
                                        src.ctypes.data, ctypes.byref(n)), "dg_mhd_regrid_plan")
        return lev, ijk, src

    def regrid(self, w, wmean=None, marks=None, **mark_args):
        """One regrid step: marks (computed unless given), plan, a new Solver on
        the new leaves with the same parameters, and the remapped state.
        Returns (solver, w_new, wmean_new)."""
        import torch
        if marks is None:
            marks, _ = self.amr_marks(w, wmean, **mark_args)
        lev, ijk, src = self.regrid_plan(marks)
        prm = {k: getattr(self.params, k) for k, _ in Params._fields_}
        new = Solver(self.dim, None, self.degree, self.divb, gamma=self.gamma, box_len=self.box_len,
                     levels=lev, ijk=ijk, **prm)
        wn, wmn = new.alloc_state(w.device)
        src_d = torch.as_tensor(src, device=w.device)
        _check(lib().dg_mhd_remap(self.h, new.h, _ptr(src_d), _ptr(w), _ptr(wmean), _ptr(wn), _ptr(wmn), _stream()),
               "dg_mhd_remap")
        new.regrid_src = src
        return new, wn, wmn

    def divb_norms(self, w, wmean=None, per_cell=False):
        """Divergence diagnostics (App. C): dict with the global norm, mean and
        maximum normalised divergence, maximum |signed divergence| and, with
        per_cell, the device rows (|div B|_K, (div B)_K, normalised)."""
        import torch
        res = torch.zeros(4, dtype=torch.float64, device=w.device)
        pc = torch.zeros((3, self.stride), dtype=torch.float64, device=w.device) if per_cell else None
        _check(lib().dg_mhd_divb(self.h, _ptr(w), _ptr(wmean), _ptr(res), _ptr(pc), _stream()), "dg_mhd_divb")
        r = res.cpu().tolist()
        out = {"total": r[0], "normalized_mean": r[1], "normalized_max": r[2], "signed_max": r[3]}
        if per_cell:
            out["per_cell"] = pc
        return out

    def limiter_counts(self, reset=False):
        p, f, l = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().dg_mhd_limiter_counts(self.h, ctypes.byref(p), ctypes.byref(f), ctypes.byref(l),
                                           1 if reset else 0), "dg_mhd_limiter_counts")
        return {"passes": p.value, "flagged": f.value, "limited": l.value}

    def status(self, sync=True, timeout_s=None):
        """The context's status word (dg_mhd_status). With timeout_s, the
        stream is first waited for by the watchdog (`wait`), so a stream that
        does not finish raises DG_E_TIMEOUT instead of blocking the host."""
        if sync and timeout_s is not None:
            wait(timeout_s=timeout_s)
        return lib().dg_mhd_status(self.h, 1 if sync else 0)
