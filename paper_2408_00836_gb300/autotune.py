"""Autotuners: the tile size of the dense sweeps (log2 amplitudes per tile,
the planner's fusion depth: a larger tile lets a sweep fuse more factors),
and the engine with its launch shape (the library's choice, the on-chip and
row engines at each CTA size, the dense sweeps at each tile).  Timing uses
CUDA events on the current stream after warm-up; candidates an engine
refuses are skipped."""

from __future__ import annotations

import numpy as np

from . import C64, ENGINE_ONCHIP, ENGINE_ROWS, Ansatz, HubError


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
                    tiles=(11, 12, 13), threads=(256, 512, 1024), reps: int = 3, warmup: int = 2):
    """Engine and launch shape for one call kind: times the library's own
    choice; the on-chip engine and the row engine (HUB_FLAG_ROWS) at each
    CTA size in `threads` (ans_set_threads; the on-chip kernel takes 256 and
    512); and the dense sweeps (HUB_FLAG_SWEEPS) at each tile in `tiles`,
    each on workspaces of the size that engine needs.  Returns (best,
    {name: ms per call}) where best is a dict of the call flags (``rows``,
    ``sweeps``), the tile and the CTA size (left set on the ansatz).
    Candidates an engine refuses are skipped."""
    import torch
    from . import workspace_tensor
    dev = torch.device("cuda", torch.cuda.current_device())
    E = torch.empty(batch, dtype=torch.float64, device=dev)
    g = torch.empty((batch, ans.P), dtype=torch.float64, device=dev)
    th = torch.tensor(np.zeros((batch, ans.P)) if theta is None else theta, dtype=torch.float64, device=dev)
    # (name, call flags, tile, (engine, threads) override or None)
    cands = [("auto", {}, 0, None)]
    cands += [(f"onchip_t{t}", {}, 0, (ENGINE_ONCHIP, t)) for t in threads if t in (256, 512)]
    cands += [(f"rows_t{t}", {"rows": True}, 0, (ENGINE_ROWS, t)) for t in threads]
    cands += [(f"sweeps_tile{k}", {"sweeps": True}, k, None) for k in tiles if k <= ans.n]
    times, picks = {}, {}

    def reset():
        ans.set_threads(dtype, ENGINE_ONCHIP, 0)
        ans.set_threads(dtype, ENGINE_ROWS, 0)

    for name, fl, k, ov in cands:
        try:
            reset()
            ans.set_tile(dtype, k)
            if ov is not None:
                ans.set_threads(dtype, *ov)
            _, eng = ans.workspace(which, dtype, batch, **fl)
            if ov is not None and eng != ov[0]:
                continue                       # that engine does not take this call
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
            picks[name] = (fl, k, ov, eng)
            del psi, lam
        except HubError:
            continue
    reset()
    if not times:
        ans.set_tile(dtype, 0)
        return {"rows": False, "sweeps": False, "tile": 0, "threads": 0, "engine": None}, times
    best = min(times, key=times.get)
    fl, k, ov, eng = picks[best]
    ans.set_tile(dtype, k)
    if ov is not None:
        ans.set_threads(dtype, *ov)
    return {"rows": bool(fl.get("rows")), "sweeps": bool(fl.get("sweeps")), "tile": k,
            "threads": ov[1] if ov else 0, "engine": ["on-chip", "rows", "sweeps"][eng], "name": best}, times
