"""Tile-size autotuner: times one call kind for each candidate tile size
(log2 amplitudes per tile, the planner's fusion depth: a larger tile lets a
sweep fuse more factors) and keeps the fastest.  Timing uses CUDA events on
the current stream after warm-up; candidates whose tile does not fit in
shared memory are skipped."""

from __future__ import annotations

import numpy as np

from . import C64, Ansatz, HubError


def autotune(ans: Ansatz, dtype: int = C64, batch: int = 1, which: int = 1,
             candidates=(11, 12, 13, 14), reps: int = 3, warmup: int = 2, theta=None):
    """Returns (best_log2_tile, {log2_tile: ms per call}) and leaves the best
    tile set on the ansatz.  ``which``: 0 energy, 1 energy + gradient."""
    import torch
    td = torch.complex64 if dtype == C64 else torch.complex128
    dev = torch.device("cuda", torch.cuda.current_device())
    psi = torch.empty((batch, 1 << ans.n), dtype=td, device=dev)
    lam = torch.empty_like(psi) if which == 1 else None
    E = torch.empty(batch, dtype=torch.float64, device=dev)
    g = torch.empty((batch, ans.P), dtype=torch.float64, device=dev)
    th = torch.tensor(np.zeros((batch, ans.P)) if theta is None else theta, dtype=torch.float64, device=dev)

    def call():
        if which == 1:
            ans.energy_grad(th, psi, lam, E, g, dtype=dtype, batch=batch)
        else:
            ans.energy(th, psi, E, dtype=dtype, batch=batch)

    times = {}
    for k in candidates:
        if k > ans.n:
            continue
        try:
            ans.set_tile(dtype, k)
            for _ in range(warmup):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            times[k] = e0.elapsed_time(e1) / reps
        except HubError:
            continue
    if not times:
        ans.set_tile(dtype, 0)
        return 0, times
    best = min(times, key=times.get)
    ans.set_tile(dtype, best)
    return best, times


def autotune_engine(ans: Ansatz, dtype: int = C64, batch: int = 1, which: int = 1, theta=None,
                    tiles=(11, 12, 13), reps: int = 3, warmup: int = 2):
    """Engine and tile choice for one call kind: times the library's own
    choice, the row engine (HUB_FLAG_ROWS), and the dense sweeps
    (HUB_FLAG_SWEEPS) at each tile in `tiles`, each on workspaces of the
    size that engine needs, and returns (best, {name: ms per call}) where
    best is a dict of the call flags (``rows``, ``sweeps``) and the tile
    (left set on the ansatz).  Candidates an engine refuses are skipped."""
    import torch
    from . import workspace_tensor
    dev = torch.device("cuda", torch.cuda.current_device())
    E = torch.empty(batch, dtype=torch.float64, device=dev)
    g = torch.empty((batch, ans.P), dtype=torch.float64, device=dev)
    th = torch.tensor(np.zeros((batch, ans.P)) if theta is None else theta, dtype=torch.float64, device=dev)
    cands = [("auto", {}, 0), ("rows", {"rows": True}, 0)]
    cands += [(f"sweeps_tile{k}", {"sweeps": True}, k) for k in tiles if k <= ans.n]
    times, engines = {}, {}
    for name, fl, k in cands:
        try:
            ans.set_tile(dtype, k)
            _, eng = ans.workspace(which, dtype, batch, **fl)
            if name == "rows" and eng != 1:
                continue                       # the row engine does not take this call
            psi = workspace_tensor(ans, which, dtype, batch, device=dev, **fl)
            lam = workspace_tensor(ans, which, dtype, batch, device=dev, **fl) if which == 1 else None

            def call():
                if which == 1:
                    ans.energy_grad(th, psi, lam, E, g, dtype=dtype, batch=batch, **fl)
                else:
                    ans.energy(th, psi, E, dtype=dtype, batch=batch, **fl)

            for _ in range(warmup):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) / reps
            engines[name] = (fl, k, eng)
            del psi, lam
        except HubError:
            continue
    if not times:
        ans.set_tile(dtype, 0)
        return {"rows": False, "sweeps": False, "tile": 0, "engine": None}, times
    best = min(times, key=times.get)
    fl, k, eng = engines[best]
    ans.set_tile(dtype, k)
    return {"rows": bool(fl.get("rows")), "sweeps": bool(fl.get("sweeps")), "tile": k,
            "engine": ["on-chip", "rows", "sweeps"][eng], "name": best}, times
