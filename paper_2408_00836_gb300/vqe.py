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
        # workspaces of the size the call's engine needs (ans.workspace)
        from . import workspace_tensor
        self.psi = workspace_tensor(ans, 1, dtype, batch, device=dev, sweeps=sweeps, rows=rows)
        self.lam = workspace_tensor(ans, 1, dtype, batch, device=dev, sweeps=sweeps, rows=rows)
        self.ckpt = torch.empty((batch, 1 << n), dtype=td, device=dev) if ckpt else None
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


def save_state(path, state: dict):
    """Writes an L-BFGS iteration state (from lbfgs_steps' on_iter) to an
    .npz file: the point, its value and gradient, the curvature pairs, the
    value history and the iteration count."""
    P = len(state["x"])
    np.savez(path, x=state["x"], f=state["f"], g=state["g"], it=state["it"],
             S=np.array(state["S"]).reshape(-1, P), Y=np.array(state["Y"]).reshape(-1, P),
             hist=np.array(state["hist"]))


def load_state(path) -> dict:
    """The state save_state wrote, for lbfgs_steps(..., resume=state)."""
    z = np.load(path)
    return {"x": z["x"], "f": float(z["f"]), "g": z["g"], "it": int(z["it"]), "S": list(z["S"]),
            "Y": list(z["Y"]), "hist": list(z["hist"])}


def lbfgs(fun, x0, max_iter=1000, m=10, e_tol=1e-7, g_tol=1e-6, c1=1e-4, max_ls=30, resume=None, on_iter=None):
    """Minimise fun(x) -> (f, grad) by L-BFGS (two-loop recursion) with a
    backtracking line search (Armijo condition); stops as in Sec. 2.1.
    resume / on_iter: as lbfgs_steps."""
    gen = lbfgs_steps(x0, max_iter, m, e_tol, g_tol, c1, max_ls, resume=resume, on_iter=on_iter)
    x = next(gen)
    try:
        while True:
            x = gen.send(fun(x))
    except StopIteration as stop:
        return stop.value


def lbfgs_steps(x0, max_iter=1000, m=10, e_tol=1e-7, g_tol=1e-6, c1=1e-4, max_ls=30, resume=None,
                on_iter=None):
    """L-BFGS as a generator: yields each point it needs evaluated, receives
    (f, grad) there, and returns (x, f, g, iterations, reason, history).
    Several of these run side by side in multistart(), whose every round is
    one batched evaluation of all their requested points.  on_iter(state)
    is called after every accepted step with the iteration state (x, f, g,
    curvature pairs S and Y, history, iteration count); resume=state
    continues from such a state (save_state / load_state), taking the same
    steps the uninterrupted run would."""
    if resume is None:
        x = np.array(x0, dtype=np.float64)
        f, g = yield x
        S, Y, hist = [], [], [f]
        it0 = 0
    else:
        x, f, g = np.array(resume["x"], dtype=np.float64), float(resume["f"]), np.array(resume["g"])
        S, Y, hist = [np.array(v) for v in resume["S"]], [np.array(v) for v in resume["Y"]], list(resume["hist"])
        it0 = int(resume["it"])
    reason = "max_iter"
    it = it0
    for it in range(it0 + 1, max_iter + 1):
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
            fn, gn = yield xn
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
        if on_iter is not None:
            on_iter({"x": x, "f": f, "g": g, "S": list(S), "Y": list(Y), "hist": list(hist), "it": it})
        if df < e_tol:
            reason = "energy"
            break
    return x, f, g, it, reason, hist


def multistart(evaluate, starts, max_iter=1000, **kw):
    """L-BFGS from several starts at once (Sec. 2.1: ten independent
    optimisations from random starts, the lowest energy kept).  evaluate(X)
    takes a [B, P] array and returns ([B] values, [B, P] gradients) -- one
    batched library call; each round evaluates every run's next requested
    point (a finished run re-evaluates its final point).  Returns a list of
    (x, f, g, iterations, reason, history), one per start."""
    starts = np.asarray(starts, dtype=np.float64)
    B = starts.shape[0]
    gens = [lbfgs_steps(starts[b], max_iter, **kw) for b in range(B)]
    req = [next(gn) for gn in gens]
    done = [None] * B
    while any(d is None for d in done):
        F, G = evaluate(np.stack(req))
        for b in range(B):
            if done[b] is not None:
                continue
            try:
                req[b] = gens[b].send((float(F[b]), G[b]))
            except StopIteration as stop:
                done[b] = stop.value
                req[b] = done[b][0]
    return done


def run_multistart(ans: Ansatz, starts, dtype: int = C64, max_iter: int = 200, use_graph: bool = True):
    """Energy-based VQE from B starts in one batched, graph-captured call per
    round; returns the VQEResult of every start (the paper keeps the
    lowest)."""
    starts = np.asarray(starts, dtype=np.float64)
    fn = EnergyGradGraph(ans, dtype=dtype, batch=starts.shape[0], use_graph=use_graph)
    t0 = time.perf_counter()
    res = multistart(lambda X: fn(X), starts, max_iter=max_iter)
    sec = time.perf_counter() - t0
    return [VQEResult(x, f, float(np.max(np.abs(g))), it, fn.evals, reason, hist, sec)
            for (x, f, g, it, reason, hist) in res]


def paper_starts(n_starts: int, P: int, seed: int = 0) -> np.ndarray:
    """Random starts of Sec. 2.1: N(0, variance 1e-5) per parameter."""
    return np.random.default_rng(seed).normal(0.0, np.sqrt(1e-5), (n_starts, P))


def warm_start_vqe(ans_u0: Ansatz, ans: Ansatz, starts, dtype: int = C64, max_iter: int = 200):
    """The warm start of Sec. 2.1: optimise the non-interacting model (U = 0,
    ans_u0: same lattice and ansatz) from the given starts, then start the
    interacting optimisation (ans) from those parameters.  Both ansatze'
    initial states must be set.  Returns (U = 0 results, interacting
    results); the paper keeps the lowest interacting energy."""
    r0 = run_multistart(ans_u0, starts, dtype=dtype, max_iter=max_iter)
    r1 = run_multistart(ans, np.stack([r.theta for r in r0]), dtype=dtype, max_iter=max_iter)
    return r0, r1


class OverlapGrad:
    """f = log10(1 - F) of Eq. 5 and its gradient through overlap_grad, on
    static buffers (psi_ref: one reference for the batch)."""

    def __init__(self, ans: Ansatz, psi_ref, dtype: int = C64, batch: int = 1):
        import torch
        self.torch = torch
        self.ans, self.dtype, self.batch = ans, dtype, batch
        td = torch.complex64 if dtype == C64 else torch.complex128
        dev = torch.device("cuda", torch.cuda.current_device())
        self.ref = psi_ref.to(device=dev, dtype=td).reshape(1, -1).contiguous()
        self.theta = torch.zeros((batch, ans.P), dtype=torch.float64, device=dev)
        self.psi = torch.empty((batch, 1 << ans.n), dtype=td, device=dev)
        self.lam = torch.empty_like(self.psi)
        self.F = torch.zeros(batch, dtype=torch.float64, device=dev)
        self.f = torch.zeros_like(self.F)
        self.g = torch.zeros((batch, ans.P), dtype=torch.float64, device=dev)
        self.evals = 0

    def __call__(self, theta):
        torch = self.torch
        self.theta.copy_(torch.from_numpy(np.asarray(theta, dtype=np.float64).reshape(self.batch, -1)))
        self.ans.overlap_grad(self.theta, self.ref, self.psi, self.lam, self.F, self.f, self.g,
                              dtype=self.dtype, batch=self.batch)
        self.evals += 1
        return self.f.cpu().numpy(), self.g.cpu().numpy(), self.F.cpu().numpy()


def run_overlap_vqe(ans: Ansatz, psi_ref, starts, dtype: int = C64, max_iter: int = 200):
    """Overlap-based optimisation (Eq. 5): minimise f = log10(1 - F) with
    F = |<psi(theta)|psi_ref>|^2 from B starts at once; returns per start
    (theta, f, F, iterations, reason)."""
    starts = np.asarray(starts, dtype=np.float64)
    fn = OverlapGrad(ans, psi_ref, dtype=dtype, batch=starts.shape[0])
    res = multistart(lambda X: fn(X)[:2], starts, max_iter=max_iter)
    F = fn(np.stack([r[0] for r in res]))[2]
    return [(r[0], r[1], float(F[b]), r[3], r[4]) for b, r in enumerate(res)]


def run_vqe(ans: Ansatz, theta0, dtype: int = C64, max_iter: int = 200, ckpt: bool = False,
            use_graph: bool = True, checkpoint_path=None, resume_path=None) -> VQEResult:
    """Energy-based VQE (Sec. 2.1) for one parameter set (batch 1): the
    ansatz's initial state must have been set with state_prepare.
    checkpoint_path: the optimiser state is written there after every step;
    resume_path: continue a run from such a file."""
    fn = EnergyGradGraph(ans, dtype=dtype, batch=1, ckpt=ckpt, use_graph=use_graph)

    def fun(x):
        E, g = fn(x)
        return float(E[0]), g[0]

    t0 = time.perf_counter()
    resume = load_state(resume_path) if resume_path else None
    on_iter = (lambda st: save_state(checkpoint_path, st)) if checkpoint_path else None
    x, f, g, it, reason, hist = lbfgs(fun, theta0, max_iter=max_iter, resume=resume, on_iter=on_iter)
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
    ap.add_argument("--checkpoint", default=None,
                    help="write the optimiser state to <path>.<dtype>.npz after every step")
    ap.add_argument("--resume", default=None, help="continue from <path>.<dtype>.npz written by --checkpoint")
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
        r = run_vqe(ans, theta0, dtype=dt, max_iter=args.iters,
                    checkpoint_path=f"{args.checkpoint}.{name}.npz" if args.checkpoint else None,
                    resume_path=f"{args.resume}.{name}.npz" if args.resume else None)
        out[name] = {"energy": r.energy, "grad_max": r.grad_norm, "iterations": r.iterations,
                     "evaluations": r.evaluations, "reason": r.reason, "seconds": round(r.seconds, 2),
                     "evals_per_s": round(r.evaluations / r.seconds, 3), "E_first": r.history[0]}
        torch.cuda.empty_cache()
    if "c64" in out and "c128" in out:
        out["final_energy_diff"] = abs(out["c64"]["energy"] - out["c128"]["energy"])
    print(json.dumps(out))


if __name__ == "__main__":
    _main()
