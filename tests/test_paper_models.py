"""The paper's other application models through the GPU library, against the
CPU oracle (same seeded inputs, element by element).

* Rayleigh damping (§3.1, eqs. (Cprop), (MatrixAA)): a chain in physical
  coordinates, with a non-normal A0 whose eigenvector matrix is far from
  unitary; the seed's f(X0) against the corrected closed form, traces and
  gradients against the oracle, FP64 and mixed.
* Ex. 3 (§4): Algorithm 2's network of 200 agents, the rank-4 change with
  B_l != B_r at two consecutive agents, the stable part of the 40 x 40 grid
  (negative parameters included): the whole sweep on both paths, sampled
  against the oracle.
Tolerances: traces 1e-10 (FP64) / 1e-8 (mixed) relative; gradients 1e-8 /
1e-6 relative to the largest component.
"""
import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err
from workloads import workload_ex3, workload_rayleigh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ly.build()
    return ly.Context(0)


def test_rayleigh_chain(ctx):
    p, vs = workload_rayleigh(masses=60, count=24)
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    st = seed.stats()
    K, M = p.meta["K"], np.diag(p.meta["masses"])
    a, b = p.meta["alpha"], p.meta["beta"]
    Ki = np.linalg.inv(K)
    X11 = np.linalg.inv(a * K + b * K @ np.linalg.solve(M, K)) + 0.5 * a * Ki @ M @ Ki + 0.5 * b * Ki
    X22 = np.linalg.inv(a * M + b * K)
    f0 = np.trace(X11) + np.trace(X22)
    assert rel_err(st["f0"], f0) <= 1e-10
    assert st["cond_Q"] > 2 * p.n  # far from unitary, unlike the modal chains
    sel = vs[::4]
    ref = np.array([oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, v) for v in sel])
    f64, i64 = seed.trace_EX(sel, return_info=True, precision=ly.FP64)
    f16, i16 = seed.trace_EX(sel, return_info=True, precision=ly.BF16_IR)
    assert all(i["status"] == 0 for i in i64 + i16)
    assert rel_err(f64, ref).max() <= 1e-10
    assert rel_err(f16, ref).max() <= 1e-8
    for prec, tg in ((ly.FP64, 1e-8), (ly.BF16_IR, 1e-6)):
        f, g = seed.grad(sel[:2], precision=prec)
        for i, v in enumerate(sel[:2]):
            fo, go = oracle.gradient(p.A0, p.U, p.V, p.G, p.E, v)
            assert np.abs(g[i] - go).max() <= tg * np.abs(go).max()


def test_rayleigh_chain_dense_similarity(ctx):
    p, vs = workload_rayleigh(masses=60, count=24, dense=True)
    ps, _ = workload_rayleigh(masses=60, count=24)
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f16 = seed.trace_EX(vs, precision=ly.BF16_IR)
    ref = np.array([oracle.trace_EX(ps.A0, ps.U, ps.V, ps.G, ps.E, v) for v in vs[:3]])
    assert rel_err(f16[:3], ref).max() <= 1e-8


@pytest.mark.parametrize("k_index", [41, 201])
def test_ex3_multi_agent_sweep(ctx, k_index):
    p, vs = workload_ex3(k_index)
    assert (vs < 0).any()  # negative parameters are part of the grid
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f16, i16 = seed.trace_EX(vs, return_info=True, precision=ly.BF16_IR)
    f64, i64 = seed.trace_EX(vs, return_info=True, precision=ly.FP64)
    assert all(i["status"] == 0 for i in i16) and all(i["status"] == 0 for i in i64)
    assert rel_err(f16, f64).max() <= 1e-8
    rng = np.random.default_rng(k_index)
    idx = np.concatenate([[0, len(vs) - 1], rng.choice(len(vs), 6, replace=False),
                          [int(np.argmax(f64))]])  # the largest H2 value: nearest to instability
    ref = np.array([oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, vs[i]) for i in idx])
    assert rel_err(f64[idx], ref).max() <= 1e-10
    assert rel_err(f16[idx], ref).max() <= 1e-8
