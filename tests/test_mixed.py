"""Mixed-precision path: the tcgen05 GEMM, the tensor-core operator, and the
refined traces and gradients against the CPU oracle.

Tolerances:
  * GEMM: |D - A B^T| <= 2^-13 |A| |B|^T elementwise (two-term BF16 split,
    FP32 accumulation: about 16 significant bits per product);
  * operator: ||T~ w - T w|| <= 1e-4 ||T w|| per system;
  * float-float residual kernel: ||T_ff w - T w|| <= 1e-12 ||T w|| per
    system (about 48 significant bits per product; the sums run over n
    terms), unchanged under power-of-two rescaling of w;
  * integer-sliced tensor-core residual kernel: the same bound (8 digits of
    6 bits per operand, exact integer sums; about 2^-47 of |A||B|^T);
  * traces after refinement: 1e-8 relative to the oracle;
  * gradients after refinement: 1e-6 relative to the largest component.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err
from workloads import workload_precision, workload_small_fp64

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def ctx():
    ly.build()
    return ly.Context(0)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 300, 150), (1600, 260, 1600)])
def test_tc_gemm_against_fp64(M, N, K):
    import torch

    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(N, K, device="cuda", generator=g, dtype=torch.float32)
    D = ly.test_tc_gemm(A, B).double()
    ref = B.double() @ A.double().T
    bound = (B.double().abs() @ A.double().abs().T) * 2.0**-13
    assert torch.all((D - ref).abs() <= bound), float(((D - ref).abs() / bound).max())


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


@pytest.mark.parametrize("adjoint", [False, True])
def test_tensor_core_operator_matches_fp64_operator(ctx, adjoint):
    import torch

    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((7, p.k, p.n, 2))
    v = torch.tensor(vs[:7], dtype=torch.float64, device="cuda")
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    y64 = ly.test_apply(seed, v, wt, ly.FP64, adjoint).cpu().numpy()
    y16 = ly.test_apply(seed, v, wt, ly.BF16_IR, adjoint).cpu().numpy()
    for b in range(7):
        assert np.linalg.norm(y16[b] - y64[b]) <= 1e-4 * np.linalg.norm(y64[b])


def test_mixed_small_chain_full_sweep(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, info = seed.trace_EX(vs, return_info=True, precision=ly.BF16_IR)
    ref = oracle.sweep(p, vs)
    assert rel_err(f, ref).max() <= TOL_MIXED
    assert all(i["status"] == 0 for i in info)
    assert all(i["refine_steps"] >= 1 for i in info)


@pytest.mark.parametrize("n,k", [(37, 3), (70, 8), (9, 1)])
def test_mixed_general_problems(ctx, n, k):
    A0, U, V, G, E, vs = random_problem(20 + n, n, k, 4)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f = seed.trace_EX(vs, precision=ly.BF16_IR)
    ref = np.array([oracle.trace_EX(A0, U, V, G, E, v) for v in vs])
    assert rel_err(f, ref).max() <= TOL_MIXED


def test_mixed_gradient(ctx):
    A0, U, V, G, E, vs = random_problem(33, 37, 3, 5)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f, g, info = seed.grad(vs[:4], return_info=True, precision=ly.BF16_IR)
    for i, v in enumerate(vs[:4]):
        fo, go = oracle.gradient(A0, U, V, G, E, v)
        assert rel_err(f[i], fo) <= TOL_MIXED
        assert np.abs(g[i] - go).max() <= 1e-6 * np.abs(go).max()


def test_mixed_full_size_precision_workload_sampled(ctx):
    """800-state chain, all 1000 parameter pairs in the bench configuration;
    sampled outputs against the oracle, all outputs against the FP64 path."""
    p, vs = workload_precision()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f16, info = seed.trace_EX(vs, return_info=True, precision=ly.BF16_IR)
    f64 = seed.trace_EX(vs, precision=ly.FP64)
    assert all(i["status"] == 0 for i in info)
    assert rel_err(f16, f64).max() <= TOL_MIXED
    # 20 spread-out parameter pairs against the oracle (it shares nothing
    # with either GPU path, unlike the FP64 comparison above)
    idx = np.linspace(0, len(vs) - 1, 20).astype(int)
    ps, _ = workload_precision(dense=False)  # f is invariant under the similarity
    ref = np.array([oracle.trace_EX(ps.A0, ps.U, ps.V, ps.G, ps.E, vs[i]) for i in idx])
    assert rel_err(f16[idx], ref).max() <= TOL_MIXED
    assert rel_err(f64[idx], ref).max() <= 1e-10


def test_mixed_with_tsvd_preconditioner(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, info = seed.trace_EX(vs[::3], return_info=True, precision=ly.BF16_IR, pbar=20)
    ref = oracle.sweep(p, vs[::3])
    assert rel_err(f, ref).max() <= TOL_MIXED
    A0, U, V, G, E, vs2 = random_problem(44, 37, 3, 5)
    s2 = ly.Seed(ctx, A0, U, V, G, E)
    f2, g2 = s2.grad(vs2[:3], precision=ly.BF16_IR, pbar=20)
    for i, v in enumerate(vs2[:3]):
        fo, go = oracle.gradient(A0, U, V, G, E, v)
        assert rel_err(f2[i], fo) <= TOL_MIXED
        assert np.abs(g2[i] - go).max() <= 1e-6 * np.abs(go).max()


@pytest.mark.parametrize("adjoint", [False, True])
def test_float_float_operator_matches_fp64_operator(ctx, adjoint):
    import torch

    p, vs = workload_small_fp64()
    A0, U, V, G, E, vs2 = random_problem(55, 70, 8, 3)
    for A0_, U_, V_, G_, E_, vv in ((p.A0, p.U, p.V, p.G, p.E, vs), (A0, U, V, G, E, vs2)):
        seed = ly.Seed(ctx, A0_, U_, V_, G_, E_)
        n, k = U_.shape
        rng = np.random.default_rng(2)
        w = rng.standard_normal((9, k, n, 2))
        v = torch.tensor(vv[:9], dtype=torch.float64, device="cuda")
        for scale in (1.0, 2.0**-700, 2.0**400, 1e-30):
            wt = torch.tensor(w * scale, dtype=torch.float64, device="cuda")
            y64 = ly.test_apply(seed, v, wt, ly.FP64, adjoint).cpu().numpy()
            yff = ly.test_apply(seed, v, wt, ly.TEST_FF, adjoint).cpu().numpy()
            assert np.isfinite(yff).all()
            for b in range(9):
                assert np.linalg.norm(yff[b] - y64[b]) <= 1e-12 * np.linalg.norm(y64[b]), (scale, b)


def test_float_float_operator_at_converged_solution(ctx):
    """At the solution T W = P the kernel output must reproduce P to the
    accuracy the refinement asks for (refine_tol 1e-11)."""
    import torch

    p, vs = workload_precision()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    W, _ = seed.param_solve(vs[:16], precision=ly.FP64)
    v = torch.tensor(vs[:16], dtype=torch.float64, device="cuda")
    wt = torch.tensor(np.stack([W.real, W.imag], axis=-1), dtype=torch.float64, device="cuda")
    y64 = ly.test_apply(seed, v, wt, ly.FP64, False).cpu().numpy()
    yff = ly.test_apply(seed, v, wt, ly.TEST_FF, False).cpu().numpy()
    for b in range(16):
        assert np.linalg.norm(yff[b] - y64[b]) <= 1e-13 * np.linalg.norm(y64[b])


def test_mixed_residual_arithmetic_options_agree(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    ref = oracle.sweep(p, vs[::4])
    for resid in (ly.RESID_FF, ly.RESID_FP64):
        f, info = seed.trace_EX(vs[::4], return_info=True, precision=ly.BF16_IR, residual=resid)
        assert rel_err(f, ref).max() <= TOL_MIXED
        assert all(i["status"] == 0 and i["rel_resid"] <= 1e-11 for i in info)


@pytest.mark.parametrize("adjoint", [False, True])
def test_sliced_tensor_core_operator_matches_fp64_operator(ctx, adjoint):
    import torch

    p, vs = workload_small_fp64()
    A0, U, V, G, E, vs2 = random_problem(56, 70, 8, 3)
    for A0_, U_, V_, G_, E_, vv in ((p.A0, p.U, p.V, p.G, p.E, vs), (A0, U, V, G, E, vs2)):
        seed = ly.Seed(ctx, A0_, U_, V_, G_, E_)
        n, k = U_.shape
        rng = np.random.default_rng(3)
        w = rng.standard_normal((9, k, n, 2))
        v = torch.tensor(vv[:9], dtype=torch.float64, device="cuda")
        for scale in (1.0, 2.0**-700, 2.0**400, 1e-30):
            wt = torch.tensor(w * scale, dtype=torch.float64, device="cuda")
            y64 = ly.test_apply(seed, v, wt, ly.FP64, adjoint).cpu().numpy()
            ytc = ly.test_apply(seed, v, wt, ly.TEST_TC, adjoint).cpu().numpy()
            assert np.isfinite(ytc).all()
            for b in range(9):
                assert np.linalg.norm(ytc[b] - y64[b]) <= 1e-12 * np.linalg.norm(y64[b]), (scale, b)


def test_sliced_tensor_core_operator_at_converged_solution(ctx):
    import torch

    p, vs = workload_precision()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    W, _ = seed.param_solve(vs[:70], precision=ly.FP64)
    v = torch.tensor(vs[:70], dtype=torch.float64, device="cuda")
    wt = torch.tensor(np.stack([W.real, W.imag], axis=-1), dtype=torch.float64, device="cuda")
    y64 = ly.test_apply(seed, v, wt, ly.FP64, False).cpu().numpy()
    ytc = ly.test_apply(seed, v, wt, ly.TEST_TC, False).cpu().numpy()
    # the digits are scaled per row of the Cauchy matrix: an entry 2^j times
    # smaller than its row's largest keeps 48 - j bits. On this chain the
    # rows span about 2^5, so the bound is 5e-13, still 20x below the
    # refinement tolerance 1e-11 that the residual is compared with.
    for b in range(70):
        assert np.linalg.norm(ytc[b] - y64[b]) <= 5e-13 * np.linalg.norm(y64[b])


def test_mixed_with_sliced_residual(ctx):
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    ref = oracle.sweep(p, vs[::4])
    f, info = seed.trace_EX(vs[::4], return_info=True, precision=ly.BF16_IR, residual=ly.RESID_TC)
    assert rel_err(f, ref).max() <= TOL_MIXED
    assert all(i["status"] == 0 and i["rel_resid"] <= 1e-11 for i in info)


def test_injected_device_wait_times_out_and_context_survives(ctx):
    """LYAP_INJECT_DEVICE_WAIT: the tensor-core GEMM issues no copy, its
    bounded mbarrier wait runs out, the kernel releases TMEM and returns, and
    the call reports LYAP_EDEVICE_TIMEOUT. The next normal call on the same
    seed and context still matches the oracle."""
    A0, U, V, G, E, vs = random_problem(41, 37, 3, 4)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    with pytest.raises(ly.LyapError) as e:
        seed.trace_EX(vs[:3], precision=ly.BF16_IR, inject=ly.INJECT_DEVICE_WAIT, maxit=20, max_refine=2)
    assert e.value.code == ly.EDEVICE_TIMEOUT
    f = seed.trace_EX(vs[:3], precision=ly.BF16_IR)
    ref = np.array([oracle.trace_EX(A0, U, V, G, E, v) for v in vs[:3]])
    assert rel_err(f, ref).max() <= TOL_MIXED
    with pytest.raises(ly.LyapError) as e:
        seed.grad(vs[:2], precision=ly.BF16_IR, inject=ly.INJECT_DEVICE_WAIT, maxit=20, max_refine=2)
    assert e.value.code == ly.EDEVICE_TIMEOUT
    f, g = seed.grad(vs[:2], precision=ly.BF16_IR)
    for i, v in enumerate(vs[:2]):
        fo, go = oracle.gradient(A0, U, V, G, E, v)
        assert rel_err(f[i], fo) <= TOL_MIXED
        assert np.abs(g[i] - go).max() <= 1e-6 * np.abs(go).max()


def test_injected_maxit_in_the_mixed_path(ctx):
    A0, U, V, G, E, vs = random_problem(42, 37, 3, 4)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f, info = seed.trace_EX(vs[:3], return_info=True, precision=ly.BF16_IR, inject=ly.INJECT_FORCE_MAXIT,
                            s=0, pbar=0, max_refine=2)
    assert all(i["status"] == ly.ENOCONV for i in info)


@pytest.mark.parametrize("n,k", [(1100, 2), (2100, 3)])
def test_sliced_operator_in_k_chunks(ctx, n, k):
    """2n above 2046: the integer-sliced product runs K in chunks whose
    exact FP32 sums are added in float-float (2 and 3 chunks here); same
    1e-12 bound against the FP64 operator, and a refined solve against the
    oracle."""
    import torch

    A0, U, V, G, E, vs = random_problem(70 + n, n, k, 2)
    seed = ly.Seed(ctx, A0, U, V, G, None)
    rng = np.random.default_rng(n)
    w = rng.standard_normal((5, k, n, 2))
    v = torch.tensor(vs[:5], dtype=torch.float64, device="cuda")
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    for adjoint in (False, True):
        y64 = ly.test_apply(seed, v, wt, ly.FP64, adjoint).cpu().numpy()
        ytc = ly.test_apply(seed, v, wt, ly.TEST_TC, adjoint).cpu().numpy()
        for b in range(5):
            assert np.linalg.norm(ytc[b] - y64[b]) <= 1e-12 * np.linalg.norm(y64[b]), (adjoint, b)
    if n == 1100:
        f, info = seed.trace_EX(vs[:3], return_info=True, precision=ly.BF16_IR, residual=ly.RESID_TC)
        assert all(i["status"] == 0 for i in info)
        ref = np.array([oracle.trace_EX(A0, U, V, G, np.eye(n), x) for x in vs[:2]])
        assert rel_err(f[:2], ref).max() <= TOL_MIXED


def symmetric_problem(seed, n, k, g):
    """A0 = Q diag(lam) Q^T made exactly symmetric, so the seed's
    eigen-decomposition is exactly real."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = -rng.uniform(0.05, 3.0, n)
    A0 = (Q * lam) @ Q.T
    A0 = (A0 + A0.T) / 2
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    E = E @ E.T / n
    vs = rng.uniform(0.2, 2.0, (24, k))
    return A0, U, V, G, E, vs


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("n,k", [(70, 3), (130, 2)])
def test_real_cauchy_layout_on_complex_vectors(ctx, n, k, adjoint):
    """With an exactly real eigen-decomposition the mixed path multiplies by
    the real n x n Cauchy matrix and takes the real and imaginary parts of
    each panel column as two columns. Complex inputs (as complex recycled
    vectors make them) must still give T(v) w: the tcgen05 operator within
    1e-4 and the integer-sliced residual within 1e-12 of the FP64 operator.
    n = 130 spans two 128-row tiles with a ragged tail."""
    import torch

    A0, U, V, G, E, vs = symmetric_problem(n + k, n, k, 4)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    assert seed.stats()["real_path"] == 1
    rng = np.random.default_rng(5)
    w = rng.standard_normal((9, k, n, 2))
    v = torch.tensor(vs[:9], dtype=torch.float64, device="cuda")
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    y64 = ly.test_apply(seed, v, wt, ly.FP64, adjoint).cpu().numpy()
    y16 = ly.test_apply(seed, v, wt, ly.BF16_IR, adjoint).cpu().numpy()
    ytc = ly.test_apply(seed, v, wt, ly.TEST_TC, adjoint).cpu().numpy()
    for b in range(9):
        nb = np.linalg.norm(y64[b])
        assert np.linalg.norm(y16[b] - y64[b]) <= 1e-4 * nb, b
        assert np.linalg.norm(ytc[b] - y64[b]) <= 1e-12 * nb, b
        # the imaginary part of the output is not zero: the Im columns count
        assert np.linalg.norm(y64[b][..., 1]) > 0.1 * nb


def test_mixed_symmetric_seed_against_the_oracle(ctx):
    """Two calls on one symmetric seed (the second starts from the first's
    recycled space) against the oracle, traces and gradients."""
    A0, U, V, G, E, vs = symmetric_problem(11, 90, 3, 5)
    seed = ly.Seed(ctx, A0, U, V, G, E)
    f1 = seed.trace_EX(vs[:12], precision=ly.BF16_IR)
    f2, g2 = seed.grad(vs[12:], precision=ly.BF16_IR)
    for i, v in enumerate(vs):
        fo = oracle.trace_EX(A0, U, V, G, E, v)
        f = f1[i] if i < 12 else f2[i - 12]
        assert rel_err(f, fo) <= TOL_MIXED, i
    for i in (0, 5, 11):
        _, go = oracle.gradient(A0, U, V, G, E, vs[12 + i])
        assert np.abs(np.asarray(g2[i]) - go).max() <= 1e-6 * np.abs(go).max(), i
