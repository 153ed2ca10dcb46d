"""Time loop with dynamic regridding of octree meshes.

Sec. 5 (adaptive mesh refinement) lets the mesh follow the solution: between
time steps, leaves whose smoothness indicator S_a(u) exceeds 2 S~ are refined
and sibling groups whose restriction has S_a(u) < S~/2 are merged, with the
L2 prolongation / restriction of the state. `evolve_amr` interleaves the
library's SSP-RK steps with those regrid steps (marks, plan, new context,
remap: Solver.regrid); a regrid whose plan keeps every leaf keeps the context,
its face lists and its buffers. Host orchestration only: every step of the
arithmetic runs in the library.
"""
from __future__ import annotations

import time


def evolve_amr(sol, w, wm, steps, regrid_every, fields=(0, 5, 6, 7), s_tilde=0.03, min_level=0, max_level=17,
               sync_timing=False):
    """Advances (sol, w, wm) by `steps` SSP-RK steps, regridding before every
    step n > 0 with n % regrid_every == 0 (regrid_every 0: never). Returns the
    final (solver, w, wmean) and a history: one record per regrid check with
    the step, the leaves before and after, the refined leaves and coarsened
    groups, whether the mesh changed and (sync_timing) the host wall time of
    the regrid."""
    history = []
    for n in range(steps):
        if regrid_every and n > 0 and n % regrid_every == 0:
            t0 = time.perf_counter()
            marks, _ = sol.amr_marks(w, wm, fields, s_tilde, min_level, max_level)
            mk = marks.cpu()
            lev, _, src = sol.regrid_plan(mk)
            rec = {"step": n, "cells_before": sol.ncell, "refined": int((mk == 1).sum()),
                   "coarsened_groups": int((mk == -1).sum()) >> sol.dim}
            unchanged = len(lev) == sol.ncell and not (src[:, 0] != 0).any()
            if not unchanged:
                sol, w, wm = sol.regrid(w, wm, marks=mk)
            rec.update(cells_after=sol.ncell, changed=not unchanged)
            if sync_timing:
                import torch
                torch.cuda.synchronize()
                rec["wall_ms"] = (time.perf_counter() - t0) * 1e3
            history.append(rec)
        sol.step(w, wm)
    return sol, w, wm, history
