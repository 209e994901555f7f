"""Pins for the CPU oracle: facts fixed by the paper or by mathematics.

Each pin is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or conjugate, a transposed operand) fails at least one
of them; the mutation tests at the end plant such mistakes in the oracle and
check that they are caught.
"""
import json
import math
import os
import types
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.lyap_oracle as ol
from workloads import haar_orthogonal, workload_small_fp64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_stable(rng, n, margin=0.5):
    R = rng.standard_normal((n, n))
    shift = np.linalg.eigvals(R).real.max() + margin
    return R - shift * np.eye(n)


# ----------------------------------------------------------------- closed forms
@pytest.mark.parametrize("method", ["kron", "bs"])
@pytest.mark.parametrize("omega,c", [(1.7, 0.3), (0.2, 0.05), (5.0, 2.0), (1.0, 1.9)])
def test_single_oscillator_modal(method, omega, c):
    # A = [[0, w], [-w, -c]]: X = [[1/c + c/(2w^2), 1/(2w)], [1/(2w), 1/c]]
    A = np.array([[0.0, omega], [-omega, -c]])
    X = ol.lyap_solve(A, np.eye(2), method)
    Xc = np.array([[1 / c + c / (2 * omega**2), 1 / (2 * omega)], [1 / (2 * omega), 1 / c]])
    np.testing.assert_allclose(X, Xc, rtol=1e-13, atol=1e-14 * np.abs(Xc).max())
    assert math.isclose(oracle.trace_product(np.eye(2), X), 2 / c + c / (2 * omega**2), rel_tol=1e-13)


@pytest.mark.parametrize("method", ["kron", "bs"])
@pytest.mark.parametrize("kk,c", [(1.0, 0.3), (4.0, 0.1), (0.25, 3.0)])
def test_single_oscillator_physical(method, kk, c):
    # A = [[0, 1], [-k, -c]]: trace X = (c^2 + (k+1)^2) / (2 c k)
    A = np.array([[0.0, 1.0], [-kk, -c]])
    X = ol.lyap_solve(A, np.eye(2), method)
    assert math.isclose(np.trace(X), (c**2 + (kk + 1) ** 2) / (2 * c * kk), rel_tol=1e-13)
    Xc12 = 1 / (2 * kk)
    assert math.isclose(X[0, 1], Xc12, rel_tol=1e-13)


@pytest.mark.parametrize("a0,u,v,vr,g,e", [(-1.0, 1.0, 0.5, 2.0, 3.0, 0.7), (-0.1, 2.0, 0.3, 0.4, 1.0, 1.0)])
def test_scalar(a0, u, v, vr, g, e):
    # n = 1: a = a0 - u v vr, 2 a x = -g^2 -> f = e g^2 / (2 |a|) for a < 0
    a = a0 - u * v * vr
    assert a < 0
    f = oracle.trace_EX(np.array([[a0]]), np.array([[u]]), np.array([[vr]]), np.array([[g]]), np.array([[e]]), [v])
    assert math.isclose(f, e * g * g / (2 * abs(a)), rel_tol=1e-14)


def test_paper_seed_closed_form_X0():
    """Paper §3.1's closed-form X0 for the modal chain (Q = I/n); its (1,1)
    coefficient is printed as 3 alpha/2 but the equation gives 1/alpha + alpha/2."""
    spec = json.load(open(os.path.join(GOLDEN, "modal_seed_X0.json")))
    for case in spec["cases"]:
        alpha = case["alpha"]
        om = np.array(case["omega"])
        m = om.size
        n = 2 * m
        A0p = np.zeros((n, n))
        A0p[:m, m:] = np.diag(om)
        A0p[m:, :m] = -np.diag(om)
        A0p[m:, m:] = -alpha * np.diag(om)
        Q = np.eye(n) / n
        # paper convention A0 X + X A0^T = -Q is the oracle's equation with A = A0^T
        X = ol.lyap_bartels_stewart(A0p.T, Q)
        c12 = -0.5
        c22 = 1 / alpha
        c11 = 1 / alpha + alpha / 2
        np.testing.assert_allclose(np.diag(X[:m, m:]) * n * om, c12, rtol=1e-12)
        np.testing.assert_allclose(np.diag(X[m:, m:]) * n * om, c22, rtol=1e-12)
        np.testing.assert_allclose(np.diag(X[:m, :m]) * n * om, c11, rtol=1e-12)
        assert not np.allclose(np.diag(X[:m, :m]) * n * om, 1.5 * alpha)  # the printed entry
        off = X.copy()
        for blk in (np.s_[:m, :m], np.s_[:m, m:], np.s_[m:, :m], np.s_[m:, m:]):
            off[blk] -= np.diag(np.diag(X[blk]))
        assert np.abs(off).max() < 1e-12 * np.abs(X).max()


def test_paper_seed_closed_form_X0_partial_modes():
    """Paper §3.1's closed-form X0 for Q = eq. (matrix Z) (the first s modes);
    the same (1,1) correction as for Q = I/n, and zero on the other modes."""
    spec = json.load(open(os.path.join(GOLDEN, "modal_seed_X0_Z.json")))
    for case in spec["cases"]:
        alpha, s = case["alpha"], case["s"]
        om = np.array(case["omega"])
        m = om.size
        n = 2 * m
        A0p = np.zeros((n, n))
        A0p[:m, m:] = np.diag(om)
        A0p[m:, :m] = -np.diag(om)
        A0p[m:, m:] = -alpha * np.diag(om)
        Q = np.zeros((n, n))
        Q[np.arange(s), np.arange(s)] = Q[m + np.arange(s), m + np.arange(s)] = 1.0 / (2 * s)
        X = ol.lyap_bartels_stewart(A0p.T, Q)
        Xc = np.zeros((n, n))
        i = np.arange(s)
        Xc[i, i] = (1 / alpha + alpha / 2) / om[:s]
        Xc[i, m + i] = Xc[m + i, i] = -0.5 / om[:s]
        Xc[m + i, m + i] = 1 / (alpha * om[:s])
        Xc /= 2 * s
        assert np.abs(X - Xc).max() <= 1e-12 * np.abs(Xc).max()
        assert not np.isclose(X[0, 0] * 2 * s * om[0], 1.5 * alpha)  # the printed entry


def test_rayleigh_seed_closed_form_X0():
    """Paper §3.1's closed-form X0 for Rayleigh damping in physical
    coordinates with Q = diag(K^-1, M^-1); the printed blocks are corrected
    (see the fixture), and the printed form is shown not to solve the equation."""
    spec = json.load(open(os.path.join(GOLDEN, "rayleigh_seed_X0.json")))
    for case in spec["cases"]:
        m, a, b = case["m"], case["alpha"], case["beta"]
        rng = np.random.default_rng(case["seed"])
        F = rng.standard_normal((m, m))
        K = F @ F.T + m * np.eye(m)
        F = rng.standard_normal((m, m))
        M = F @ F.T + m * np.eye(m)
        Ki, Mi = np.linalg.inv(K), np.linalg.inv(M)
        Z = np.zeros((2 * m, 2 * m))
        Z[:m, :m], Z[m:, m:] = Ki, Mi
        A0p = np.block([[np.zeros((m, m)), np.eye(m)], [-Mi @ K, -a * np.eye(m) - b * Mi @ K]])
        X = ol.lyap_bartels_stewart(A0p.T, Z)  # paper convention A0 X + X A0^T = -Z
        S = np.linalg.inv(a * K + b * K @ Mi @ K)
        X11 = S + 0.5 * a * Ki @ M @ Ki + 0.5 * b * Ki
        X22 = np.linalg.inv(a * M + b * K)
        Xc = np.block([[X11, -0.5 * Ki], [-0.5 * Ki, X22]])
        assert np.abs(X - Xc).max() <= 1e-12 * np.abs(Xc).max()
        Xp = np.block([[S + a * Ki @ Mi @ Ki + b * Ki, -0.5 * Ki], [-0.5 * Ki, S]])  # as printed
        assert np.abs(X - Xp).max() > 1e-2 * np.abs(Xc).max()
    # one mass: X11 = 1/(c k) + c/(2 k^2), X22 = 1/c with c = alpha + beta k
    k, a, b = 2.5, 0.3, 0.05
    c = a + b * k
    X = ol.lyap_bartels_stewart(np.array([[0.0, 1.0], [-k, -c]]).T, np.diag([1 / k, 1.0]))
    np.testing.assert_allclose(X, [[1 / (c * k) + c / (2 * k * k), -0.5 / k], [-0.5 / k, 1 / c]], rtol=1e-13)


def test_modal_chain_seed_trace_full_size():
    """f(X0) = sum_i (2/alpha + alpha/2)/omega_i for the decoupled modal seed
    (G = E = I), at the full 100-state chain; and continuity as v -> 0+."""
    p, _ = workload_small_fp64()
    om = p.meta["omega"]
    alpha = p.meta["alpha"]
    closed = math.fsum((2 / alpha + alpha / 2) / om)
    f0 = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, [0.0, 0.0])
    assert math.isclose(f0, closed, rel_tol=1e-12)
    f_small = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, [1e-9, 1e-9])
    assert math.isclose(f_small, closed, rel_tol=1e-6)


# ------------------------------------------------------- brute force and exact
EXACT_CASES = [
    [[-2, 1], [0, -3]],
    [[-3, 1, 0], [-1, -2, 1], [0, 2, -4]],
    [[-5, 1, 0, 2], [0, -3, 1, 0], [1, 0, -4, 1], [-2, 0, 1, -6]],
]


@pytest.mark.parametrize("A", EXACT_CASES)
def test_exact_rational(A):
    n = len(A)
    C = [[int(i == j) + (1 if abs(i - j) == 1 else 0) for j in range(n)] for i in range(n)]
    Xe = ol.lyap_exact(A, C)
    # verify the exact solution satisfies the equation exactly
    for i in range(n):
        for j in range(n):
            s = sum(Fraction(A[l][i]) * Xe[l][j] + Xe[i][l] * Fraction(A[l][j]) for l in range(n))
            assert s == -C[i][j]
    Xf = np.array([[float(x) for x in row] for row in Xe])
    An = np.array(A, dtype=float)
    Cn = np.array(C, dtype=float)
    for method in ("kron", "bs"):
        np.testing.assert_allclose(ol.lyap_solve(An, Cn, method), Xf, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_bartels_stewart_vs_kronecker(n):
    rng = np.random.default_rng(n)
    A = random_stable(rng, n)
    G = rng.standard_normal((n, 2))
    C = G @ G.T
    np.testing.assert_allclose(ol.lyap_bartels_stewart(A, C), ol.lyap_kron(A, C), rtol=1e-11, atol=1e-13)


def test_brute_force_parametrized_tiny():
    """Whole pipeline (A(v), G G^T, trace) at n = 6 against the Kronecker form."""
    rng = np.random.default_rng(7)
    n, k = 6, 2
    A0 = random_stable(rng, n, margin=2.0)
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, 3))
    E = rng.standard_normal((n, n))
    E = E @ E.T
    v = np.array([0.7, 1.3])
    f_kron = oracle.trace_EX(A0, U, V, G, E, v, method="kron")
    f_bs = oracle.trace_EX(A0, U, V, G, E, v, method="bs")
    A = A0 - U @ np.diag(v) @ V.T
    # brute force without the oracle's helpers
    K = np.kron(np.eye(n), A.T) + np.kron(A.T, np.eye(n))
    X = np.linalg.solve(K, -(G @ G.T).flatten("F")).reshape(n, n, order="F")
    f_direct = float(np.sum(E * X))
    assert math.isclose(f_kron, f_direct, rel_tol=1e-12)
    assert math.isclose(f_bs, f_direct, rel_tol=1e-11)


# ----------------------------------------------------------------- invariants
def _random_problem(rng, n=30, k=3, g=4):
    A0 = random_stable(rng, n, margin=1.0)
    U = rng.standard_normal((n, k)) * 0.2
    V = rng.standard_normal((n, k)) * 0.2
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    E = E @ E.T / n
    v = rng.uniform(0.2, 2.0, k)
    return A0, U, V, G, E, v


def test_orthogonal_similarity_invariance():
    rng = np.random.default_rng(11)
    A0, U, V, G, E, v = _random_problem(rng)
    S = haar_orthogonal(rng, A0.shape[0])
    f1 = oracle.trace_EX(A0, U, V, G, E, v)
    f2 = oracle.trace_EX(S @ A0 @ S.T, S @ U, S @ V, S @ G, S @ E @ S.T, v)
    assert math.isclose(f1, f2, rel_tol=1e-11)


def test_scaling_of_G():
    rng = np.random.default_rng(12)
    A0, U, V, G, E, v = _random_problem(rng)
    f1 = oracle.trace_EX(A0, U, V, G, E, v)
    f3 = oracle.trace_EX(A0, U, V, 3.0 * G, E, v)
    assert math.isclose(f3, 9.0 * f1, rel_tol=1e-12)


def test_duality():
    """trace(E X) = trace(G G^T Y) with A Y + Y A^T = -E."""
    rng = np.random.default_rng(13)
    A0, U, V, G, E, v = _random_problem(rng)
    A = oracle.param_matrix(A0, U, V, v)
    X = ol.lyap_bartels_stewart(A, G @ G.T)
    Y = ol.lyap_bartels_stewart(A.T, E)
    assert math.isclose(oracle.trace_product(E, X), oracle.trace_product(G @ G.T, Y), rel_tol=1e-11)


def test_symmetry_psd_backward_error():
    p, vs = workload_small_fp64()
    for v in vs[::17]:
        A = oracle.param_matrix(p.A0, p.U, p.V, v)
        f, X = oracle.solve(p.A0, p.U, p.V, p.G, p.E, v)
        d = oracle.check_solution(A, p.G @ p.G.T, X)
        assert d["asym"] < 1e-12
        assert d["backward_error"] < 1e-14
        assert d["min_eig_rel"] > 0  # G = I: X positive definite
        assert f > 0


def test_against_scipy_lapack():
    rng = np.random.default_rng(14)
    A0, U, V, G, E, v = _random_problem(rng, n=40)
    A = oracle.param_matrix(A0, U, V, v)
    X = ol.lyap_bartels_stewart(A, G @ G.T)
    Xs = sla.solve_continuous_lyapunov(A.T, -G @ G.T)
    np.testing.assert_allclose(X, Xs, rtol=1e-10, atol=1e-12 * np.abs(Xs).max())


# ------------------------------------------------------------------- gradient
def test_gradient_central_differences():
    rng = np.random.default_rng(15)
    A0, U, V, G, E, v = _random_problem(rng, n=24, k=3)
    f, g = oracle.gradient(A0, U, V, G, E, v)
    h = 1e-6
    for i in range(v.size):
        vp = v.copy()
        vm = v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (oracle.trace_EX(A0, U, V, G, E, vp) - oracle.trace_EX(A0, U, V, G, E, vm)) / (2 * h)
        assert math.isclose(g[i], fd, rel_tol=1e-6, abs_tol=1e-9 * abs(f))


def test_gradient_scalar_closed_form():
    # f = e g^2 / (2 (u v vr - a0)) for a = a0 - u v vr < 0 -> df/dv = -e g^2 u vr / (2 (u v vr - a0)^2)
    a0, u, vr, g, e, v = -1.0, 1.5, 0.8, 2.0, 0.5, 0.4
    f, grad = oracle.gradient(np.array([[a0]]), np.array([[u]]), np.array([[vr]]), np.array([[g]]), np.array([[e]]), [v])
    d = u * v * vr - a0
    assert math.isclose(grad[0], -e * g * g * u * vr / (2 * d * d), rel_tol=1e-13)


# ---------------------------------------------------- planted mistakes (CPU)
class _NoConj(types.SimpleNamespace):
    pass


def _numpy_without_conj():
    ns = _NoConj(**{name: getattr(np, name) for name in dir(np) if not name.startswith("__")})
    ns.conj = lambda x: x
    return ns


def test_mutation_dropped_conjugate_is_caught(monkeypatch):
    monkeypatch.setattr(ol, "np", _numpy_without_conj())
    A = np.array([[0.0, 1.7], [-1.7, -0.3]])
    X = ol.lyap_bartels_stewart(A, np.eye(2))
    assert not math.isclose(np.trace(X), 2 / 0.3 + 0.3 / (2 * 1.7**2), rel_tol=1e-6)


def test_mutation_dropped_parameter_term_is_caught(monkeypatch):
    monkeypatch.setattr(ol, "param_matrix", lambda A0, U, V, v: np.asarray(A0, dtype=float))
    f = ol.trace_EX(np.array([[-1.0]]), np.array([[1.0]]), np.array([[2.0]]), np.array([[3.0]]), np.array([[0.7]]), [0.5])
    assert not math.isclose(f, 0.7 * 9 / (2 * 2.0), rel_tol=1e-6)


def test_mutation_transposed_operand_is_caught(monkeypatch):
    # solving A X + X A^T instead of A^T X + X A: the entries of the modal
    # oscillator's X (not its trace) expose it
    real = ol.lyap_bartels_stewart
    monkeypatch.setattr(ol, "lyap_bartels_stewart", lambda A, C: real(np.asarray(A).T, C))
    A = np.array([[0.0, 1.7], [-1.7, -0.3]])
    X = ol.lyap_solve(A, np.eye(2), "bs")
    assert not math.isclose(X[0, 1], 1 / (2 * 1.7), rel_tol=1e-6)


def test_mutation_wrong_sign_is_caught(monkeypatch):
    real = ol.lyap_kron
    monkeypatch.setattr(ol, "lyap_kron", lambda A, C: -real(A, C))
    A = np.array([[0.0, 1.0], [-4.0, -0.1]])
    X = ol.lyap_solve(A, np.eye(2), "kron")
    assert not math.isclose(np.trace(X), (0.01 + 25) / (2 * 0.1 * 4), rel_tol=1e-6)
