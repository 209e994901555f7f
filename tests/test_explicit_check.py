"""The independent explicit check (lyap_check_explicit): X(v) formed from
the seed's eigen-decomposition and a capacitance solution, and the true
residual A(v)^T X + X A(v) + G G^T evaluated in FP64 from the caller's
matrices. Converged solutions (FP64 path and refined mixed path) have a
backward error at rounding level (<= 1e-12) and their explicit trace equals
lyap_trace_EX and the oracle (1e-10); a perturbed solution is caught."""
import math

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err
from workloads import workload_rayleigh

pytestmark = pytest.mark.gpu


def _problem(seed, n, k, g):
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((n, n)) / math.sqrt(n)
    A0 = R - (np.linalg.eigvals(R).real.max() + 1.0) * np.eye(n)
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    return A0, U, V, G, E @ E.T / n, rng.uniform(0.2, 2.0, (4, k))


@pytest.mark.parametrize("precision", [ly.FP64, ly.BF16_IR])
def test_explicit_check_of_converged_solutions(precision):
    ly.build()
    ctx = ly.Context(0)
    for A0, U, V, G, E, vs in (_problem(91, 37, 3, 5),):
        seed = ly.Seed(ctx, A0, U, V, G, E)
        W, info = seed.param_solve(vs, precision=precision)
        be, tr = ly.check_explicit(seed, vs, W, A0, U, V, G, E)
        f = seed.trace_EX(vs, precision=precision)
        ref = np.array([oracle.trace_EX(A0, U, V, G, E, v) for v in vs])
        assert (be <= 1e-12).all(), be
        assert rel_err(tr, f).max() <= 1e-10
        assert rel_err(tr, ref).max() <= 1e-10
        # a solution off by 1e-6 relative shows in the residual
        Wp = W * (1.0 + 1e-6)
        be2, _ = ly.check_explicit(seed, vs, Wp, A0, U, V, G, E)
        assert (be2 > 1e-9).all(), be2
    # physical coordinates: a non-normal A0 with an ill-conditioned eigenbasis
    p, vs = workload_rayleigh(masses=30, count=4)
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    W, _ = seed.param_solve(vs, precision=precision)
    be, tr = ly.check_explicit(seed, vs, W, p.A0, p.U, p.V, p.G, p.E)
    assert (be <= 1e-11).all(), be
    ref = np.array([oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, v) for v in vs])
    assert rel_err(tr, ref).max() <= 1e-9
