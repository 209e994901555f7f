"""The batched Nelder-Mead driver (paper §4, Ex. 1 uses MATLAB's fminsearch)
on plain functions, without a GPU: it converges on a bowl and on
Rosenbrock's valley, and, started from the same simplex with the same
stopping rule, it takes the same iterates as scipy's Nelder-Mead (the
fminsearch algorithm): evaluating the four trial points of an iteration in
one batch changes which values are computed, not the path."""
import numpy as np
from scipy.optimize import minimize

from paper_2312_08201_gb300.optimize import _fminsearch_simplex, nelder_mead_batched


def rosen(x):
    return 100.0 * (x[1] - x[0] ** 2) ** 2 + (1.0 - x[0]) ** 2


def test_bowl():
    c = np.array([0.3, -1.2, 2.0])
    x, f, info = nelder_mead_batched(lambda X: ((X - c) ** 2).sum(axis=1) + 3.0, np.zeros(3), 1e-8, 1e-12)
    assert info["converged"] and np.abs(x - c).max() < 1e-6 and abs(f - 3.0) < 1e-10
    # calls are batches: at most 1 + (iterations) + (shrinks) library calls
    assert info["calls"] <= 1 + 2 * info["iterations"]


def test_same_path_as_scipy_nelder_mead():
    x0 = np.array([-1.2, 1.0])
    x, f, info = nelder_mead_batched(lambda X: np.array([rosen(r) for r in X]), x0, 1e-10, 1e-10, max_iter=2000)
    r = minimize(rosen, x0, method="Nelder-Mead",
                 options=dict(initial_simplex=_fminsearch_simplex(x0), xatol=1e-10, fatol=1e-10, maxiter=2000,
                              maxfev=100000))
    assert info["converged"] and np.abs(x - 1.0).max() < 1e-8
    assert np.allclose(x, r.x, rtol=0, atol=1e-12)
    assert abs(info["iterations"] - r.nit) <= 1  # scipy counts its loop from 1
