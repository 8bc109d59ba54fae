"""The VQE driver's optimiser state: an L-BFGS run interrupted after a few
steps and resumed from the saved file (save_state / load_state) takes the
same steps as the uninterrupted run (host only, no GPU)."""

import numpy as np

from paper_2408_00836_gb300 import vqe


def _fun(x):
    # a smooth non-quadratic test function (a chain of Rosenbrock valleys
    # plus a small quartic), value and gradient
    a, b = x[:-1], x[1:]
    f = np.sum(100.0 * (b - a * a) ** 2 + (1.0 - a) ** 2) + 0.01 * np.sum(x ** 4)
    g = np.zeros_like(x)
    g[:-1] += -400.0 * a * (b - a * a) - 2.0 * (1.0 - a)
    g[1:] += 200.0 * (b - a * a)
    g += 0.04 * x ** 3
    return float(f), g


def test_interrupted_lbfgs_resumes_on_the_same_path(tmp_path):
    x0 = np.random.default_rng(3).uniform(-1.0, 1.0, 12)
    full = vqe.lbfgs(_fun, x0, max_iter=60, e_tol=0.0, g_tol=0.0)
    path = tmp_path / "state.npz"
    part = vqe.lbfgs(_fun, x0, max_iter=25, e_tol=0.0, g_tol=0.0,
                     on_iter=lambda st: vqe.save_state(path, st))
    assert part[3] == 25
    st = vqe.load_state(path)
    assert st["it"] == 25 and np.array_equal(st["x"], part[0])
    rest = vqe.lbfgs(_fun, None, max_iter=60, e_tol=0.0, g_tol=0.0, resume=st)
    assert rest[3] == full[3] == 60
    assert np.array_equal(rest[0], full[0])          # the same iterates, bit for bit
    assert rest[1] == full[1]
    assert rest[5] == full[5]                          # the same value history


def test_stopping_rules():
    x0 = np.random.default_rng(4).uniform(-1.0, 1.0, 6)
    _, f, g, it, reason, hist = vqe.lbfgs(_fun, x0, max_iter=500, e_tol=1e-9, g_tol=1e-30)
    assert reason == "energy" and it < 500 and abs(hist[-1] - hist[-2]) < 1e-9
    _, f, g, it, reason, hist = vqe.lbfgs(_fun, x0, max_iter=500, e_tol=0.0, g_tol=1e-3)
    assert reason == "gradient" and np.max(np.abs(g)) < 1e-3
    assert vqe.lbfgs(_fun, x0, max_iter=3, e_tol=0.0, g_tol=0.0)[4] == "max_iter"
