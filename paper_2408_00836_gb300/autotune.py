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
