"""Fault injection made on the host (nothing faults or hangs on the device): a
NaN planted in the state is reported by the status word as DG_E_NONFINITE when
the timestep of Sec. 3.6 is taken, and the synchronising read clears the word;
a negative density mean under the positivity limiter of Sec. 4.3 is floored at
eps_rho and reported as DG_W_FLOOR."""
import pytest

from oracle.dg import Scheme
from paper_1806_02343_gb300 import workloads as W

from gpu_helpers import means_to_device, to_device

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_in_the_state_is_reported(prec):
    from paper_1806_02343_gb300.binding import DG_PREC_FP32MIX, DG_PREC_FP64, Solver
    S = Scheme(3, 2, "glm", G, (5, 4, 3))
    w0 = S.project(W.SmoothFourier3D(nvar=9))
    sol = Solver(3, (5, 4, 3), 2, "glm", gamma=G, box_len=S.L,
                 precision=DG_PREC_FP32MIX if prec == "fp32" else DG_PREC_FP64)
    w = to_device(w0, sol)
    wm = means_to_device(w0, sol, S) if prec == "fp32" else None
    sol.dt(w, wm)
    assert sol.status() == 0
    w[0, 7] = float("nan")                                 # density mean of cell 7
    if wm is not None:
        wm[0, 7] = float("nan")
    sol.dt(w, wm)
    assert sol.status() == -4                              # DG_E_NONFINITE
    assert sol.status() == 0                               # read and cleared


def test_negative_density_mean_is_floored_and_reported():
    from paper_1806_02343_gb300.binding import Solver
    S = Scheme(3, 1, "glm", G, (4, 4, 4))
    w0 = S.project(W.SmoothFourier3D(nvar=9))
    w0[9, 0] = -0.1                                        # cell 9: negative density mean
    sol = Solver(3, (4, 4, 4), 1, "glm", gamma=G, box_len=S.L, positivity=1)
    w = to_device(w0, sol)
    sol.limit(w)
    assert sol.status() == 1                               # DG_W_FLOOR
    assert float(w[0, 9]) == sol.params.eps_rho
    assert sol.status() == 0
