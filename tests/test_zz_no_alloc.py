"""dg_mhd_rhs_noalloc: the operator for callers that cannot allocate device
memory (their pool owns it, or a cudaMalloc's implicit synchronisation is not
allowed where they call us). It keeps its scratch in the library's static
device array; its output must equal the context-based dg_mhd_rhs, and a second
call in a row (same shared array, reused) must give it again.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test."""
import numpy as np
import pytest

from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("D,d,divb,ncell", [(3, 2, "glm", (7, 6, 5)), (2, 2, "powell", (24, 20))])
def test_noalloc_matches_rhs_twice(D, d, divb, ncell):
    import torch
    from paper_1806_02343_gb300.binding import Solver, rhs_noalloc
    S = Scheme(D, d, divb, G, ncell)
    fn = W.SmoothFourier3D(nvar=S.V) if D == 3 else (lambda x: W.alfven_2d(x, nvar=S.V))
    w0 = S.project(fn)
    sol = Solver(D, ncell, d, divb, gamma=G, box_len=S.L)
    ch, kap = (2.7, 1.3) if divb == "glm" else (0.0, 0.0)
    if divb == "glm":
        sol.set_glm(ch, kap)
    w = torch.zeros((sol.nrows, sol.stride), dtype=torch.float64, device="cuda")
    w[:, : sol.ncell] = torch.as_tensor(w0.T.copy(), device="cuda")
    ref = torch.zeros_like(w)
    sol.rhs(w, None, ref)
    ref_np = ref[:, : sol.ncell].cpu().numpy()
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out = torch.full_like(w, float("nan"))
        rhs_noalloc(D, ncell, d, divb, w, out, gamma=G, box_len=S.L, c_h=ch, damping_rate=kap, status=status)
        torch.cuda.synchronize()
        got = out[:, : sol.ncell].cpu().numpy()
        assert _rel(got, ref_np) < 1e-12
        assert int(status.item()) == 0
    # a NaN planted in the input (on the host side of the call) reaches the
    # caller through the status word; the next clean call reports 0 again
    wbad = w.clone()
    wbad[0, 3] = float("nan")
    rhs_noalloc(D, ncell, d, divb, wbad, out, gamma=G, box_len=S.L, c_h=ch, damping_rate=kap, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    rhs_noalloc(D, ncell, d, divb, w, out, gamma=G, box_len=S.L, c_h=ch, damping_rate=kap, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert _rel(out[:, : sol.ncell].cpu().numpy(), ref_np) < 1e-12


def test_noalloc_rejects_oversized_problem():
    import torch
    from paper_1806_02343_gb300 import binding
    w = torch.zeros((90, 64 ** 3), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.DGError) as e:
        binding.rhs_noalloc(3, (64, 64, 64), 2, "glm", w, w, c_h=1.0, damping_rate=1.0)
    assert e.value.code == -1


def test_noalloc_rejects_mismatched_buffers():
    import torch
    from paper_1806_02343_gb300 import binding
    ok = torch.zeros((90, 224), dtype=torch.float64, device="cuda")   # 7 x 6 x 5 cells -> stride 224
    for bad in (torch.zeros((90, 32), dtype=torch.float64, device="cuda"),
                torch.zeros((90, 224), dtype=torch.float32, device="cuda"),
                torch.zeros((224, 90), dtype=torch.float64, device="cuda").t()):
        with pytest.raises(ValueError):
            binding.rhs_noalloc(3, (7, 6, 5), 2, "glm", ok, bad, c_h=1.0, damping_rate=1.0)
