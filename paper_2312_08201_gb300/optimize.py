"""Viscosity optimisation on top of the library (paper §4, Ex. 1).

The paper minimises the total average energy trace(X(v)) over the damper
viscosities with a Nelder-Mead search (MATLAB's fminsearch, started from
v0 = (100, 100, 100), tolerance 1e-4), evaluating every trial point with its
recycled solver. Two drivers are provided here; both are host logic around
the library's batched calls, and every function value and gradient comes
from the GPU:

* ``nelder_mead``: the simplex method with the standard coefficients
  (reflection 1, expansion 2, contraction 1/2, shrink 1/2) and fminsearch's
  initial simplex (5% steps) and stopping rule (TolX, TolFun). Each
  iteration evaluates the reflection, expansion and both contraction points
  in one library call (one lockstep batch that shares the recycled Krylov
  space), then takes the simplex decision from those values; a shrink
  evaluates its k new vertices in one call. The iterates are those of the
  one-point-at-a-time method: only unused trial values are extra.
* ``lbfgs``: a gradient method (scipy's L-BFGS-B) on the adjoint gradient
  of lyap_grad.

Both search in x = log(v): the viscosities stay positive (v_i = 0 is
excluded by §1 and negative dampers are unphysical) and the simplex steps
are relative.
"""
from __future__ import annotations

import numpy as np


def _fminsearch_simplex(x0):
    """fminsearch's initial simplex: x0 and, per coordinate, x0 with that
    coordinate scaled by 1.05 (0.00025 when it is zero)."""
    x0 = np.asarray(x0, dtype=np.float64)
    pts = [x0.copy()]
    for i in range(x0.size):
        y = x0.copy()
        y[i] = 1.05 * y[i] if y[i] != 0 else 0.00025
        pts.append(y)
    return np.array(pts)


def nelder_mead_batched(fbatch, x0, tol_x=1e-4, tol_f=1e-4, max_iter=400):
    """Minimise f with the Nelder-Mead simplex method.

    fbatch(X) returns f at each row of X (one call per batch of points).
    Returns (x_best, f_best, info) with info = dict(iterations, evaluations,
    calls, converged, history of f_best).
    """
    S = _fminsearch_simplex(x0)
    F = np.asarray(fbatch(S), dtype=np.float64)
    nd = S.shape[1]
    calls, evals, hist = 1, len(S), []
    it = 0
    converged = False
    while it < max_iter:
        order = np.argsort(F, kind="stable")
        S, F = S[order], F[order]
        hist.append(float(F[0]))
        if np.max(np.abs(S[1:] - S[0])) <= tol_x and np.max(np.abs(F[1:] - F[0])) <= tol_f:
            converged = True
            break
        it += 1
        c = S[:-1].mean(axis=0)
        worst = S[-1]
        xr = c + (c - worst)
        xe = c + 2.0 * (c - worst)
        xc = c + 0.5 * (c - worst)  # outside contraction
        xcc = c - 0.5 * (c - worst)  # inside contraction
        fr, fe, fc, fcc = np.asarray(fbatch(np.stack([xr, xe, xc, xcc])), dtype=np.float64)
        calls += 1
        evals += 4
        if fr < F[0]:
            S[-1], F[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < F[-2]:
            S[-1], F[-1] = xr, fr
        elif fr < F[-1]:
            if fc <= fr:
                S[-1], F[-1] = xc, fc
            else:
                S, F = _shrink(fbatch, S, F)
                calls += 1
                evals += nd
        else:
            if fcc < F[-1]:
                S[-1], F[-1] = xcc, fcc
            else:
                S, F = _shrink(fbatch, S, F)
                calls += 1
                evals += nd
    order = np.argsort(F, kind="stable")
    S, F = S[order], F[order]
    return S[0].copy(), float(F[0]), dict(iterations=it, evaluations=evals, calls=calls, converged=converged,
                                          history=hist)


def _shrink(fbatch, S, F):
    S = S.copy()
    S[1:] = S[0] + 0.5 * (S[1:] - S[0])
    F = F.copy()
    F[1:] = np.asarray(fbatch(S[1:]), dtype=np.float64)
    return S, F


def nelder_mead(seed, v0, tol=1e-4, max_iter=400, **opts):
    """Minimise f(v) = trace(E X(v)) over v > 0 with Nelder-Mead in log(v).

    ``seed`` is a factored Seed; ``opts`` are lyap_opts fields (e.g.
    precision). Returns (v_best, f_best, info)."""

    def fbatch(X):
        return np.asarray(seed.trace_EX(np.exp(X), **opts), dtype=np.float64)

    x, f, info = nelder_mead_batched(fbatch, np.log(np.asarray(v0, dtype=np.float64)), tol, tol, max_iter)
    return np.exp(x), f, info


def lbfgs(seed, v0, tol=1e-8, max_iter=200, **opts):
    """Minimise f(v) over v > 0 with L-BFGS-B in log(v), using the adjoint
    gradient (df/dlog v_i = v_i df/dv_i). Returns (v_best, f_best, info)."""
    from scipy.optimize import minimize

    count = [0]

    def fg(x):
        v = np.exp(x)[None, :]
        f, g = seed.grad(v, **opts)
        count[0] += 1
        return float(np.asarray(f)[0]), np.asarray(g, dtype=np.float64)[0] * v[0]

    r = minimize(fg, np.log(np.asarray(v0, dtype=np.float64)), jac=True, method="L-BFGS-B",
                 options=dict(maxiter=max_iter, gtol=tol, ftol=1e-15))
    return np.exp(r.x), float(r.fun), dict(iterations=int(r.nit), evaluations=count[0], converged=bool(r.success),
                                           message=str(r.message))
