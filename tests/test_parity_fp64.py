"""FP64 GPU path against the CPU oracle (element by element, same seeded inputs).

Tolerance: 1e-10 relative on trace(E X(v)) for the FP64 path, the bar the
library is built to; gradients 1e-8 relative against the oracle's adjoint
gradient and 1e-5 against central differences of the GPU traces.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err
from workloads import generic_dense, workload_precision, workload_small_fp64

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def ctx():
    ly.build()
    return ly.Context(0)


def random_problem(seed, n, k, g, margin=1.0):
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((n, n)) / math.sqrt(n)
    A0 = R - (np.linalg.eigvals(R).real.max() + margin) * np.eye(n)
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    E = E @ E.T / n
    vs = rng.uniform(0.2, 2.0, (12, k))
    return A0, U, V, G, E, vs


def oracle_sweep(A0, U, V, G, E, vs):
    return np.array([oracle.trace_EX(A0, U, V, G, E, v) for v in vs])


def test_small_chain_full_sweep(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, info = seed.trace_EX(vs, return_info=True)
    ref = oracle.sweep(p, vs)
    err = rel_err(f, ref)
    assert err.max() <= TOL_FP64, (err.max(), int(err.argmax()))
    assert all(i["status"] == 0 for i in info)
    assert max(i["rel_resid"] for i in info) < 1e-10
    st = seed.stats()
    # ||Qp||_F ||Qp^{-1}||_F equals n for a unitary eigenvector matrix
    assert p.n <= st["cond_Q"] < 10 * p.n and st["max_re_lambda"] < 0
    om, alpha = p.meta["omega"], p.meta["alpha"]
    assert math.isclose(st["f0"], float(np.sum((2 / alpha + alpha / 2) / om)), rel_tol=1e-12)


def test_small_chain_dense_similarity(ctx):
    p, vs = workload_small_fp64()
    pd = generic_dense(p, np.random.default_rng(5))
    seed = ly.Seed(ctx, pd.A0, pd.U, pd.V, pd.G, pd.E)
    sel = vs[::5]
    f = seed.trace_EX(sel)
    ref = oracle.sweep(p, sel)  # the similarity leaves f unchanged
    assert rel_err(f, ref).max() <= TOL_FP64


@pytest.mark.parametrize("batch", [1, 5, 0])
def test_general_problem_ragged(ctx, batch):
    # n = 37 (ragged against the 64-row tiles), k = 3, G of rank 5, E dense SPD
    A0, U, V, G, E, vs = random_problem(3, 37, 3, 5)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f, info = seed.trace_EX(vs, return_info=True, batch=batch)
    ref = oracle_sweep(A0, U, V, G, E, vs)
    assert rel_err(f, ref).max() <= TOL_FP64
    assert all(i["status"] == 0 for i in info)


@pytest.mark.parametrize("n,k", [(1, 1), (6, 1), (9, 4), (70, 8)])
def test_sizes_and_ranks(ctx, n, k):
    A0, U, V, G, E, vs = random_problem(10 + n + k, n, k, 2)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f = seed.trace_EX(vs[:5])
    ref = oracle_sweep(A0, U, V, G, E, vs[:5])
    assert rel_err(f, ref).max() <= TOL_FP64


def test_identity_E_is_default(ctx):
    A0, U, V, G, E, vs = random_problem(4, 20, 2, 3)
    seed = ly.Seed(ctx, A0, U, V, G, None)
    f = seed.trace_EX(vs[:4])
    ref = oracle_sweep(A0, U, V, G, np.eye(20), vs[:4])
    assert rel_err(f, ref).max() <= TOL_FP64


def test_gradient_against_oracle_and_fd(ctx):
    A0, U, V, G, E, vs = random_problem(6, 37, 3, 5)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f, g, info = seed.grad(vs[:4], return_info=True)
    for i, v in enumerate(vs[:4]):
        fo, go = oracle.gradient(A0, U, V, G, E, v)
        assert rel_err(f[i], fo) <= TOL_FP64
        assert np.abs(g[i] - go).max() <= 1e-8 * np.abs(go).max()
        assert info[i]["err_est"] < 1e-9
    h = 1e-6
    v = vs[0]
    for j in range(3):
        vp, vm = v.copy(), v.copy()
        vp[j] += h
        vm[j] -= h
        fp, fm = seed.trace_EX(np.stack([vp, vm]))
        fd = (fp - fm) / (2 * h)
        assert abs(g[0, j] - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(f[0]))


def test_param_solve_returns_capacitance_solution(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    W, info = seed.param_solve(vs[:3])
    assert W.shape == (3, 2, 100)
    assert np.isfinite(W).all() and all(i["status"] == 0 for i in info)


def test_edge_cases(ctx):
    A0, U, V, G, E, vs = random_problem(7, 10, 2, 2)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    assert seed.trace_EX(np.zeros((0, 2))).shape == (0,)
    bad = vs[:2].copy()
    bad[1, 0] = 0.0  # v_i = 0 is excluded (§1)
    with pytest.raises(ly.LyapError) as e:
        seed.trace_EX(bad)
    assert e.value.code == ly.EINVAL
    bad[1, 0] = np.nan
    with pytest.raises(ly.LyapError):
        seed.trace_EX(bad)
    with pytest.raises(ly.LyapError) as e:
        ly.Seed(ctx, -A0, U, V, G, E)  # unstable seed
    assert e.value.code == ly.EUNSTABLE_SEED
    with pytest.raises(ly.LyapError):
        ly.Seed(ctx, A0, np.ones((10, 9)), np.ones((10, 9)), G, E)  # k > 8


def test_injected_allocation_failure_and_maxit(ctx):
    A0, U, V, G, E, vs = random_problem(8, 12, 2, 2)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    with pytest.raises(ly.LyapError) as e:
        seed.trace_EX(vs[:2], inject=ly.INJECT_ALLOC_FAIL)
    assert e.value.code == ly.ENOMEM
    f, info = seed.trace_EX(vs[:2], return_info=True, inject=ly.INJECT_FORCE_MAXIT, s=0, pbar=0)
    # one block-Jacobi preconditioned iteration cannot reach the 1e-12
    # residual on this 24-unknown system (a TSVD of full rank would be exact)
    assert all(i["status"] == ly.ENOCONV and i["iters"] == 1 for i in info)
    assert all(i["rel_resid"] > 1e-12 for i in info)
    # the seed stays usable
    f = seed.trace_EX(vs[:2])
    assert rel_err(f, oracle_sweep(A0, U, V, G, E, vs[:2])).max() <= TOL_FP64


def test_full_size_precision_workload_sampled(ctx):
    """800-state chain, 1000 ordered parameter pairs, in the bench's launch
    configuration; four sampled outputs checked against the oracle."""
    p, vs = workload_precision()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, info = seed.trace_EX(vs, return_info=True)
    assert np.isfinite(f).all()
    assert all(i["status"] == 0 for i in info)
    idx = [0, 333, 666, 999]
    ref = np.array([oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, vs[i]) for i in idx])
    assert rel_err(f[idx], ref).max() <= TOL_FP64


@pytest.mark.parametrize("pbar", [8, 30])
def test_tsvd_preconditioner_keeps_results_and_cuts_iterations(ctx, pbar):
    """The truncated-SVD coupling of eq. (prec) changes the iteration count,
    never the answer (flexible recycled solver)."""
    p, vs = workload_small_fp64()
    sel = vs[::7]
    s0 = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f0, i0 = s0.trace_EX(sel, return_info=True, pbar=0)
    s1 = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f1, i1 = s1.trace_EX(sel, return_info=True, pbar=pbar)
    ref = oracle.sweep(p, sel)
    assert rel_err(f1, ref).max() <= TOL_FP64
    assert rel_err(f0, ref).max() <= TOL_FP64
    assert np.mean([i["iters"] for i in i1]) < np.mean([i["iters"] for i in i0])
    A0, U, V, G, E, vs2 = random_problem(9, 37, 3, 5)
    s2 = ly.Seed(ctx, A0, U, V, G, E)
    f2, g2 = s2.grad(vs2[:3], pbar=pbar)
    for i, v in enumerate(vs2[:3]):
        fo, go = oracle.gradient(A0, U, V, G, E, v)
        assert rel_err(f2[i], fo) <= TOL_FP64
        assert np.abs(g2[i] - go).max() <= 1e-8 * np.abs(go).max()
