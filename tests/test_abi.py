"""The C-ABI library loads and exports every symbol include/dg_mhd.h declares
(no compute calls: runs without a GPU). Also checks host-only entry points."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dg_mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(dg_mhd_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1806_02343_gb300 import build, binding
    build.build()
    return binding.lib()


def test_header_and_binding_agree():
    from paper_1806_02343_gb300 import binding
    assert _declared() == set(binding.EXPORTS)


def test_library_exports_all_declared(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_params_and_strerror(lib):
    from paper_1806_02343_gb300 import binding
    p = binding.default_params()
    assert p.cfl == 0.3 and p.cfl_glm == 0.9 and p.c_r == 0.18 and p.eta_powell == 0.2
    assert p.Mtilde == 5.0 and p.beta == 2.0 and p.tvb_eps == 1e-8
    assert p.eps_rho == 1e-12 and p.eps_p == 1e-12 and p.rk_order == 3
    assert lib.dg_mhd_strerror(0) == b"ok"
    assert lib.dg_mhd_strerror(-4).startswith(b"non-finite")


def test_init_rejects_bad_arguments(lib):
    import ctypes
    from paper_1806_02343_gb300 import binding
    m = binding.MeshDesc()
    m.dim = 4
    h = ctypes.c_void_p()
    assert lib.dg_mhd_init(ctypes.byref(m), 2, 0, 5.0 / 3.0, None, ctypes.byref(h)) == -2
    m.dim = 3
    m.n[0] = m.n[1] = m.n[2] = 4
    m.box_len = 1.0
    m.periodic = 1
    assert lib.dg_mhd_init(ctypes.byref(m), 7, 0, 5.0 / 3.0, None, ctypes.byref(h)) == -7
    assert lib.dg_mhd_init(ctypes.byref(m), 2, 5, 5.0 / 3.0, None, ctypes.byref(h)) == -1
    assert lib.dg_mhd_init(ctypes.byref(m), 2, 0, 1.0, None, ctypes.byref(h)) == -1
    bad = binding.default_params(rk_order=5)             # SSP-RK orders are 1..4 (0: degree + 1)
    assert lib.dg_mhd_init(ctypes.byref(m), 2, 0, 5.0 / 3.0, ctypes.byref(bad), ctypes.byref(h)) == -1
    assert lib.dg_mhd_init(None, 2, 0, 1.4, None, ctypes.byref(h)) == -1
    m.n[0] = m.n[1] = 2048
    m.n[2] = 1024                                        # 2^32 cells: beyond 32-bit indices
    assert lib.dg_mhd_init(ctypes.byref(m), 2, 0, 5.0 / 3.0, None, ctypes.byref(h)) == -2
    assert lib.dg_mhd_rhs(None, None, None, None, None, None) == -1
    assert lib.dg_mhd_step(None, None, None, None, None) == -1
    assert lib.dg_mhd_divb(None, None, None, None, None, None) == -1
    # regridding entry points: NULL contexts and arrays are DG_E_ARG before any device work
    assert lib.dg_mhd_smoothness(None, None, None, 1, None, None) == -1
    assert lib.dg_mhd_amr_marks(None, None, None, 1, 0.03, 0, 8, None, None, None) == -1
    n = ctypes.c_int64(-5)
    assert lib.dg_mhd_regrid_plan(None, None, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.dg_mhd_remap(None, None, None, None, None, None, None, None) == -1


def test_octree_mesh_validation_rejects_bad_meshes(lib):
    import ctypes
    import numpy as np
    from paper_1806_02343_gb300 import binding

    def init(leaves, D=3):
        m = binding.MeshDesc()
        m.dim = D
        m.box_len = 1.0
        m.periodic = 1
        lev = np.array([l for l, _ in leaves], dtype=np.int8)
        ijk = np.array([k for _, k in leaves], dtype=np.int32).reshape(-1)
        m.n_leaves = len(leaves)
        m.level = lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
        m.ijk = ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        return lib.dg_mhd_init(ctypes.byref(m), 1, 0, 5.0 / 3.0, None, ctypes.byref(h))

    full = [(1, k) for k in np.ndindex(2, 2, 2)]
    assert init(full[:-1]) == -2                        # incomplete cover
    assert init(full + [(2, (0, 0, 0))]) == -2          # overlap
    assert init(full + [full[0]]) == -2                 # duplicate leaf
    # unbalanced: one level-1 cell refined twice next to level-1 neighbours
    deep = [(1, k) for k in np.ndindex(2, 2, 2) if k != (0, 0, 0)]
    deep += [(2, k) for k in np.ndindex(2, 2, 2) if k != (1, 1, 1)]
    deep += [(3, tuple(2 + x for x in k)) for k in np.ndindex(2, 2, 2)]
    assert init(deep) == -2


def test_host_entry_points_reject_null_arguments(lib):
    """The context-free host calls (planning, faces, basis, regrid tables)
    return DG_E_ARG for NULL outputs or inputs and for a too-small capacity,
    and answer size queries with NULL output arrays."""
    import ctypes
    import numpy as np
    lev = np.full(4, 1, dtype=np.int8)
    ijk = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.int32)
    marks = np.zeros(4, dtype=np.int8)
    n = ctypes.c_int64()
    lp, kp, mp = lev.ctypes.data, ijk.ctypes.data, marks.ctypes.data
    assert lib.dg_mhd_regrid_plan_mesh(2, 4, lp, kp, None, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.dg_mhd_regrid_plan_mesh(2, 4, lp, kp, mp, 0, None, None, None, None) == -1
    assert lib.dg_mhd_regrid_plan_mesh(2, 4, lp, kp, mp, 0, None, None, None, ctypes.byref(n)) == 0 and n.value == 4
    out = np.zeros(3, dtype=np.int32)
    assert lib.dg_mhd_regrid_plan_mesh(2, 4, lp, kp, mp, 3, out.ctypes.data, out.ctypes.data, out.ctypes.data,
                                       ctypes.byref(n)) == -1                     # capacity 3 < 4
    assert lib.dg_mhd_sibling_groups(2, 4, lp, kp, 0, None, None) == -1
    assert lib.dg_mhd_sibling_groups(2, 4, lp, kp, 0, None, ctypes.byref(n)) == 0 and n.value == 1
    assert lib.dg_mhd_octree_faces(2, 4, None, kp, 0, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.dg_mhd_octree_faces(2, 4, lp, kp, 0, 0, None, None, None, None) == -1
    assert lib.dg_mhd_octree_faces(2, 4, lp, kp, 2, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.dg_mhd_octree_faces(2, 4, lp, kp, 0, 0, None, None, None, ctypes.byref(n)) == 0 and n.value == 8
    r, v = ctypes.c_int(), ctypes.c_int()
    assert lib.dg_mhd_basis_values(3, 2, 1, 1, None, 0, None, ctypes.byref(r), ctypes.byref(v)) == -1
    assert lib.dg_mhd_basis_values(3, 2, 1, 0, None, 0, None, None, ctypes.byref(v)) == -1
    assert lib.dg_mhd_basis_values(3, 2, 1, 0, None, 0, None, ctypes.byref(r), ctypes.byref(v)) == 0
    assert (r.value, v.value) == (90, 9)
    assert lib.dg_mhd_regrid_tables(3, 2, 0, 0, None, None) == -1
    sizes = np.zeros(6, dtype=np.int64)
    assert lib.dg_mhd_regrid_tables(3, 2, 0, 0, None, sizes.ctypes.data) == 0 and sizes[0] == 3 * 10 * 10
    small = np.zeros(1)
    assert lib.dg_mhd_regrid_tables(3, 2, 0, 1, small.ctypes.data, sizes.ctypes.data) == -1


def test_eps_hlld_and_noalloc_arguments_checked_on_host(lib):
    """NaN or out-of-range HLLD tolerances, and missing GLM speeds of the
    allocation-free operator, are rejected before any device work."""
    import ctypes
    from paper_1806_02343_gb300 import binding
    m = binding.mesh_desc(3, (4, 4, 4))
    h = ctypes.c_void_p()
    for eps in (float("nan"), -1e-8, 1.0):
        bad = binding.default_params(eps_hlld=eps)
        assert lib.dg_mhd_init(ctypes.byref(m), 2, 1, 5.0 / 3.0, ctypes.byref(bad), ctypes.byref(h)) == -1
        assert lib.dg_mhd_rhs_noalloc(ctypes.byref(m), 2, 1, 5.0 / 3.0, ctypes.byref(bad), 1.0, 1.0,
                                      ctypes.c_void_p(16), ctypes.c_void_p(16), None, None) == -1
    for ch, kap in ((0.0, 1.0), (float("nan"), 1.0), (1.0, -1.0)):
        assert lib.dg_mhd_rhs_noalloc(ctypes.byref(m), 2, 1, 5.0 / 3.0, None, ch, kap,
                                      ctypes.c_void_p(16), ctypes.c_void_p(16), None, None) == -1


def test_probe_rejects_bad_arguments_on_host(lib):
    import ctypes
    r, m = ctypes.c_double(), ctypes.c_double()
    assert lib.dg_mhd_probe(4, None, None, 0, ctypes.byref(r), ctypes.byref(m), None) == -1
    assert lib.dg_mhd_probe(-1, None, None, 0, ctypes.byref(r), ctypes.byref(m), None) == -1
    assert lib.dg_mhd_probe(3, None, None, 1 << 20, ctypes.byref(r), ctypes.byref(m), None) == -1
    assert lib.dg_mhd_probe(3, ctypes.c_void_p(16), ctypes.c_void_p(32), 100, ctypes.byref(r), ctypes.byref(m),
                            None) == -1
    assert lib.dg_mhd_probe(0, None, None, 0, None, ctypes.byref(m), None) == -1
