"""Pins of the projection-framework oracle (paper §2.2; oracle/projection.py).

Each check is fixed by the paper or by the mathematics, not by the oracle's
own formulas:
* the basis spans eq. (EK_def)'s explicit set [P, A0^-1 P, A0 P, A0^-2 P, ...]
  (compared through orthogonal projectors of an SVD of that set);
* A0 EK_m lies in EK_{m+1}: the Arnoldi relation of the backward error proof;
* the nestedness argument of §2.2: A(v)^-1 P lies in EK_1 and A(v) P in EK_2
  for every v, B_l lies in the space and B_r in general does not;
* the backward error proposition's cheap formula equals the backward error's
  definition evaluated with the full n x n residual;
* when the space fills R^n the projected solution is the exact solution
  (Bartels-Stewart of lyap_oracle) and the backward error vanishes;
* the trace identity trace(V Y V^T) = trace(Y);
* Algorithm 1 accepts v in order with non-decreasing m, meets its bound, and
  its traces agree with the exact ones within a small multiple of the bound;
* for symmetric A(v) and E = I the trace is exact on EK_1 (trace(X) =
  trace(A^-1 C) / 2 and A(v)^-1 P lies in EK_1);
* Ex. 1 case b): the dimension of the space that meets eps for the first
  equation, against the values the paper prints (tests/golden).
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import projection as pj
from workloads import generic_dense, mass_spring_chain, multi_agent, two_row_system


def chain_problem(masses: int, dampers, seed: int = 3, alpha: float = 0.04):
    rng = np.random.default_rng(seed)
    springs = rng.uniform(0.5, 2.0, masses + 1)
    return generic_dense(mass_spring_chain(springs, alpha, dampers), rng)


def setup(p):
    sq = pj.seed_quantities(p.A0, p.U, p.V, p.G, p.E)
    return sq, pj.ExtendedKrylov(sq["A0p"], sq["P"])


def projector(Q):
    return Q @ Q.T


def test_basis_spans_the_extended_krylov_set():
    p = chain_problem(20, [1, 7])
    sq, ek = setup(p)
    A, P = sq["A0p"], sq["P"]
    Ainv = np.linalg.inv(A)
    pos, neg = P.copy(), Ainv @ P
    cols = [P, neg]
    for m in range(1, 4):
        ek.ensure(m)
        Vm = ek.basis(m)
        assert np.abs(Vm.T @ Vm - np.eye(Vm.shape[1])).max() < 1e-12
        S = np.hstack(cols)
        Us, sig, _ = np.linalg.svd(S, full_matrices=False)
        Q = Us[:, sig > 1e-12 * sig[0]]
        assert Q.shape[1] == Vm.shape[1] == 4 * m * p.k
        assert np.linalg.norm(projector(Vm) - projector(Q), 2) < 1e-7
        pos, neg = A @ pos, Ainv @ neg
        cols += [pos, neg]  # next block of eq. (EK_def): A0^m P, A0^-(m+1) P


def test_arnoldi_relation():
    # The late blocks come from candidates that are nearly in the space already
    # (down to 1e-10 of their norm here), and orthogonalising them costs
    # accuracy in proportion: hence the looser bound from m = 3 on.
    p = chain_problem(20, [1, 7])
    sq, ek = setup(p)
    for m, tol in ((1, 1e-13), (2, 1e-13), (3, 1e-9), (4, 1e-9)):
        pm = pj.projected_matrices(ek, m, sq["Bl"], sq["Br"])
        Vnext = ek.blocks[m]
        AV = sq["A0p"] @ pm["Vm"]
        resid = AV - pm["Vm"] @ pm["Tm"] - Vnext @ pm["EmT"]
        assert np.linalg.norm(resid) <= tol * np.linalg.norm(AV)


def asymmetric_problem():
    """The chain with B_l != B_r (V = U + a seeded perturbation)."""
    p = chain_problem(20, [1, 7])
    rng = np.random.default_rng(5)
    p.V = p.U + 0.3 * rng.standard_normal(p.U.shape) / np.sqrt(p.n)
    return p


@pytest.mark.parametrize("v", [[0.3, 2.0], [5.0, 0.07], [1.0, 1.0]])
def test_nestedness_of_the_parametric_spaces(v):
    p = asymmetric_problem()
    sq, ek = setup(p)
    Av = sq["A0p"] - (sq["Bl"] * np.asarray(v)[None, :]) @ sq["Br"].T
    V1 = ek.basis(1)
    ek.ensure(2)
    V2 = ek.basis(2)
    W = np.linalg.solve(Av, sq["P"])
    assert np.linalg.norm(W - V1 @ (V1.T @ W)) <= 1e-10 * np.linalg.norm(W)
    Z = Av @ sq["P"]
    assert np.linalg.norm(Z - V2 @ (V2.T @ Z)) <= 1e-10 * np.linalg.norm(Z)
    assert np.linalg.norm(sq["Bl"] - V1 @ (V1.T @ sq["Bl"])) <= 1e-12 * np.linalg.norm(sq["Bl"])
    # B_r is not represented exactly (the remark after eq. (param_projected))
    assert np.linalg.norm(sq["Br"] - V1 @ (V1.T @ sq["Br"])) > 1e-3 * np.linalg.norm(sq["Br"])


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_backward_error_formula_matches_its_definition(m):
    p = chain_problem(20, [1, 7])
    sq, ek = setup(p)
    off = pj.offline_norms(sq["A0p"], sq["Bl"], sq["Br"])
    pm = pj.projected_matrices(ek, m, sq["Bl"], sq["Br"])
    for v in ([0.3, 2.0], [5.0, 0.07]):
        Y = pj.solve_projected(pm, ek.G, v)
        cheap = pj.backward_error_cheap(pm, Y, ek.G, v, off)
        full = pj.backward_error_full(sq, pm, Y, v)
        # m = 5 fills R^40: the cheap formula gives exactly 0, the definition
        # the rounding of the explicit n x n residual
        assert cheap == pytest.approx(full, rel=1e-8, abs=1e-11)


def test_projected_solution_is_exact_when_the_space_fills():
    # n = 20 = 5 blocks of 4k (k = 1): EK_5 is all of R^20
    p = chain_problem(10, [1])
    sq, ek = setup(p)
    off = pj.offline_norms(sq["A0p"], sq["Bl"], sq["Br"])
    pm = pj.projected_matrices(ek, 5, sq["Bl"], sq["Br"])
    assert pm["Vm"].shape == (20, 20) and ek.blocks[5].shape[1] == 0
    for v in ([0.5], [3.0], [0.02]):
        Y = pj.solve_projected(pm, ek.G, v)
        X = sq["X0"] + pm["Vm"] @ Y @ pm["Vm"].T
        f_exact, X_exact = oracle.solve(p.A0, p.U, p.V, p.G, p.E, v)
        assert np.linalg.norm(X - X_exact) <= 1e-9 * np.linalg.norm(X_exact)
        assert pj.backward_error_cheap(pm, Y, ek.G, v, off) == 0.0
        assert pj.trace_value(sq, pm, Y, p.E) == pytest.approx(f_exact, rel=1e-10)


def test_trace_identity():
    p = chain_problem(20, [1, 7])
    sq, ek = setup(p)
    pm = pj.projected_matrices(ek, 3, sq["Bl"], sq["Br"])
    Y = pj.solve_projected(pm, ek.G, [0.4, 1.7])
    X = pm["Vm"] @ Y @ pm["Vm"].T
    assert np.trace(X) == pytest.approx(np.trace(Y), rel=1e-12)
    # with E = I the trace value needs no basis: f0 + trace(Y)
    assert pj.trace_value(sq, pm, Y, np.eye(p.n)) == pytest.approx(sq["f0"] + np.trace(Y), rel=1e-12)


def network_problem(skew: float):
    """Agents on a graph (§3.2 data); a seeded skew-symmetric part of size
    ``skew`` makes A0 non-symmetric without changing its symmetric part
    (so it stays stable), and E is a random rank-5 PSD weight."""
    rng = np.random.default_rng(7)
    p = multi_agent(rng, agents=60, p=0.1, tunable_edges=4)
    n = p.n
    S = rng.standard_normal((n, n))
    p.A0 = p.A0 + skew * (S - S.T) / np.sqrt(n)
    R = rng.standard_normal((n, 5))
    p.E = R @ R.T / n
    vs = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(8, 4)))
    return p, vs[np.argsort(vs[:, 0])]


def test_algorithm1_sweep():
    p, vs = network_problem(skew=2.0)
    exact = np.array([oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, v) for v in vs])
    m_prev = None
    for eps in (1e-6, 1e-10):
        f, m_used, delta = pj.eksm_sweep(p.A0, p.U, p.V, p.G, p.E, vs, eps=eps, m_max=40)
        assert np.all(np.isfinite(f)) and np.all(m_used >= 1)
        assert np.all(np.diff(m_used) >= 0)  # v are accepted in order
        assert np.all(delta <= eps)
        assert 16 * m_used.max() < p.n  # converged well before the space fills R^n
        # forward error <= (condition) x backward error; the factor here is
        # modest (measured below 0.1), 100 leaves room
        assert np.max(np.abs(f - exact) / np.abs(exact)) <= 100 * eps
        if m_prev is not None:
            assert np.all(m_used >= m_prev) and m_used.sum() > m_prev.sum()
        m_prev = m_used


def test_symmetric_trace_is_exact_on_the_first_space():
    # For symmetric A(v) and E = I, trace(X_d) = trace(A(v)^-1 C) / 2 with C the
    # right-hand side, and A(v)^-1 P lies in EK_1: the Galerkin solution on
    # EK_1 already has the exact trace, although its backward error is not small.
    p, vs = network_problem(skew=0.0)
    p.E = np.eye(p.n)
    sq, ek = setup(p)
    pm = pj.projected_matrices(ek, 1, sq["Bl"], sq["Br"])
    off = pj.offline_norms(sq["A0p"], sq["Bl"], sq["Br"])
    for v in vs[:4]:
        Y = pj.solve_projected(pm, ek.G, v)
        assert pj.backward_error_cheap(pm, Y, ek.G, v, off) > 1e-8
        exact = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, v)
        assert pj.trace_value(sq, pm, Y, p.E) == pytest.approx(exact, rel=1e-12)


def two_row_x0(p, s):
    """Closed-form seed solution for Q = eq. (matrix Z) (pinned against
    Bartels-Stewart in test_oracle.py's partial-mode closed-form test)."""
    om, a, nm = p.meta["omega"], p.meta["alpha"], p.meta["omega"].size
    X = np.zeros((p.n, p.n))
    i = np.arange(s)
    X[i, i] = (1 / a + a / 2) / om[:s]
    X[i, nm + i] = X[nm + i, i] = -0.5 / om[:s]
    X[nm + i, nm + i] = 1 / (a * om[:s])
    return X / (2 * s)


@pytest.mark.slow
@pytest.mark.parametrize("case", [0, 1])
def test_ex1b_extended_krylov_dimension(case):
    """Ex. 1 case b): the space that meets eps = 1e-8 for the first equation
    has the dimension the paper prints, within two blocks of 12."""
    spec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ex1b_eksm_dimensions.json")))
    mod, ref = spec["model"], spec["printed"][case]
    p = two_row_system(mod["d"], ref["i1"], ref["i2"], 21, alpha=mod["alpha"], stiffness=tuple(mod["stiffness"]))
    X0 = two_row_x0(p, 21)
    f, m_used, delta = pj.eksm_sweep(p.A0, p.U, p.V, p.G, p.E, np.array([mod["v0"]]), eps=mod["eps"],
                                     m_max=mod["m_max"], X0=X0)
    k4 = 4 * p.k
    assert delta[0] <= mod["eps"] and np.isfinite(f[0])
    assert abs(m_used[0] * k4 - ref["dim"]) <= spec["tolerance_blocks"] * k4
