"""VQE driver: host L-BFGS over the energy and adjoint gradient, the
evaluation captured once in a CUDA graph and replayed per iteration.

The optimiser follows Sec. 2.1: L-BFGS; stop when the change of the energy
between the last two steps is below 1e-7, when the gradient (max norm) is
below 1e-6, or after ``max_iter`` steps.  Everything on the amplitudes runs
in the library's kernels; the host holds only the parameters, the L-BFGS
history and the line search.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import C64, C128, Ansatz


class EnergyGradGraph:
    """energy_grad on static buffers, captured into a CUDA graph.

    Calling the object copies theta (host) into the static device buffer,
    replays the graph and returns (E, grad) as host arrays.  The first call
    of energy_grad (done here, outside the capture) makes every allocation
    the call needs, so the captured graph contains kernel launches only.
    """

    def __init__(self, ans: Ansatz, dtype: int = C64, batch: int = 1, ckpt: bool = False,
                 use_graph: bool = True, sweeps: bool = False, rows: bool = False):
        import torch
        self.torch = torch
        self.sweeps, self.rows = sweeps, rows   # engine selection (see Ansatz.energy_grad)
        self.ans, self.dtype, self.batch = ans, dtype, batch
        td = torch.complex64 if dtype == C64 else torch.complex128
        dev = torch.device("cuda", torch.cuda.current_device())
        n = ans.n
        self.theta_h = torch.zeros((batch, ans.P), dtype=torch.float64).pin_memory()
        self.theta = torch.zeros((batch, ans.P), dtype=torch.float64, device=dev)
        self.psi = torch.empty((batch, 1 << n), dtype=td, device=dev)
        self.lam = torch.empty_like(self.psi)
        self.ckpt = torch.empty_like(self.psi) if ckpt else None
        self.E = torch.zeros(batch, dtype=torch.float64, device=dev)
        self.g = torch.zeros((batch, ans.P), dtype=torch.float64, device=dev)
        self.E_h = torch.zeros(batch, dtype=torch.float64).pin_memory()
        self.g_h = torch.zeros((batch, ans.P), dtype=torch.float64).pin_memory()
        self.graph = None
        self.evals = 0
        self._call()                        # warm-up: allocations happen here
        torch.cuda.synchronize()
        if use_graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                self._call()                # second warm-up on the capture stream
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._call()
            torch.cuda.synchronize()

    def _call(self):
        self.ans.energy_grad(self.theta, self.psi, self.lam, self.E, self.g, ckpt=self.ckpt,
                             dtype=self.dtype, batch=self.batch, sweeps=self.sweeps, rows=self.rows)

    def __call__(self, theta: np.ndarray):
        torch = self.torch
        self.theta_h.copy_(torch.from_numpy(np.asarray(theta, dtype=np.float64).reshape(self.batch, -1)))
        self.theta.copy_(self.theta_h, non_blocking=True)
        if self.graph is not None:
            self.graph.replay()
        else:
            self._call()
        self.E_h.copy_(self.E, non_blocking=True)
        self.g_h.copy_(self.g, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        self.evals += 1
        return self.E_h.numpy().copy(), self.g_h.numpy().copy()


@dataclass
class VQEResult:
    theta: np.ndarray
    energy: float
    grad_norm: float
    iterations: int
    evaluations: int
    reason: str
    history: list = field(default_factory=list)
    seconds: float = 0.0


def lbfgs(fun, x0, max_iter=1000, m=10, e_tol=1e-7, g_tol=1e-6, c1=1e-4, max_ls=30):
    """Minimise fun(x) -> (f, grad) by L-BFGS (two-loop recursion) with a
    backtracking line search (Armijo condition); stops as in Sec. 2.1."""
    x = np.array(x0, dtype=np.float64)
    f, g = fun(x)
    S, Y, hist = [], [], [f]
    reason = "max_iter"
    it = 0
    for it in range(1, max_iter + 1):
        if np.max(np.abs(g)) < g_tol:
            reason = "gradient"
            it -= 1
            break
        q = g.copy()
        alpha = []
        for s, y in reversed(list(zip(S, Y))):
            a = (s @ q) / (y @ s)
            alpha.append(a)
            q -= a * y
        if S:
            q *= (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
        for (s, y), a in zip(zip(S, Y), reversed(alpha)):
            b = (y @ q) / (y @ s)
            q += (a - b) * s
        d = -q
        gd = g @ d
        if gd >= 0:                      # not a descent direction: restart
            S, Y = [], []
            d = -g
            gd = g @ d
        step = 1.0 if S else min(1.0, 1.0 / max(np.linalg.norm(g), 1e-12))
        for _ in range(max_ls):
            xn = x + step * d
            fn, gn = fun(xn)
            if fn <= f + c1 * step * gd:
                break
            step *= 0.5
        s, y = xn - x, gn - g
        if s @ y > 1e-12:
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        df = abs(fn - f)
        x, f, g = xn, fn, gn
        hist.append(f)
        if df < e_tol:
            reason = "energy"
            break
    return x, f, g, it, reason, hist


def run_vqe(ans: Ansatz, theta0, dtype: int = C64, max_iter: int = 200, ckpt: bool = False,
            use_graph: bool = True) -> VQEResult:
    """Energy-based VQE (Sec. 2.1) for one parameter set (batch 1): the
    ansatz's initial state must have been set with state_prepare."""
    fn = EnergyGradGraph(ans, dtype=dtype, batch=1, ckpt=ckpt, use_graph=use_graph)

    def fun(x):
        E, g = fn(x)
        return float(E[0]), g[0]

    t0 = time.perf_counter()
    x, f, g, it, reason, hist = lbfgs(fun, theta0, max_iter=max_iter)
    sec = time.perf_counter() - t0
    return VQEResult(x, f, float(np.max(np.abs(g))), it, fn.evals, reason, hist, sec)


def _main():
    """Run the energy-based VQE of a seeded workload in complex64 and then in
    complex128 from the same start, and print one JSON line with both
    results (final energies, iterations, evaluations, wall time)."""
    import argparse
    import json

    import torch

    from . import PREP_SLATER, Model, hva_groups, square_lattice
    from . import workloads as W

    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--workload", type=int, default=4)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--dtypes", default="c64,c128")
    args = ap.parse_args()
    torch.cuda.init()
    w = W.workload(args.workload, batch_sets=1)
    bonds, cls = square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    ans = Ansatz(m, hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    theta0 = w.theta()[0]
    out = {"workload": w.name, "qubits": w.n_qubits, "params": ans.P, "max_iter": args.iters}
    for name in args.dtypes.split(","):
        dt = C64 if name == "c64" else C128
        ans.state_prepare(PREP_SLATER, w.orbital_perturbation(), None, None, dt, 1)
        r = run_vqe(ans, theta0, dtype=dt, max_iter=args.iters)
        out[name] = {"energy": r.energy, "grad_max": r.grad_norm, "iterations": r.iterations,
                     "evaluations": r.evaluations, "reason": r.reason, "seconds": round(r.seconds, 2),
                     "evals_per_s": round(r.evaluations / r.seconds, 3), "E_first": r.history[0]}
        torch.cuda.empty_cache()
    if "c64" in out and "c128" in out:
        out["final_energy_diff"] = abs(out["c64"]["energy"] - out["c128"]["energy"])
    print(json.dumps(out))


if __name__ == "__main__":
    _main()
