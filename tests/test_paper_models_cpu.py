"""Input generators of the paper's application models, pinned on the CPU.

* Ex. 3 (§4): Algorithm 2's graph, the agent network of §3.2, the rank-4
  change at two consecutive agents and the 40 x 40 grid reproduce the
  printed count of unstable configurations (356 of 6,400,
  tests/golden/ex3_stable_count.json); the stability test used to filter
  the grid agrees with brute-force eigenvalues.
* Rayleigh damping (§3.1): the generator's A_p(v) is eq. (MatrixAA) with
  C(v) = alpha M + beta K + B D(v) B^T, and the oracle's seed solution has
  the (corrected) closed-form trace.
"""
import json
import os

import numpy as np

import oracle
from oracle import lyap_oracle as ol
from workloads import (EX3_POSITIONS, agent_network, ex3_grid, ex3_laplacian, ex3_problem, rayleigh_chain,
                       stable_mask, workload_ex3)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ex3_unstable_count_matches_the_paper():
    spec = json.load(open(os.path.join(GOLDEN, "ex3_stable_count.json")))
    assert tuple(spec["positions_read"]) == EX3_POSITIONS
    grid = ex3_grid()
    assert grid.shape == (spec["printed"]["grid_values_per_parameter"] ** 2, 4)
    unstable = sum(int((~stable_mask(ex3_problem(200, k), grid)).sum()) for k in EX3_POSITIONS)
    assert unstable == spec["printed"]["unstable"]
    assert sum(len(workload_ex3(k)[1]) for k in EX3_POSITIONS) == spec["printed"]["stable"]


def test_ex3_graph_and_network():
    L = ex3_laplacian(200)
    assert np.array_equal(L, L.T) and np.allclose(L.sum(axis=1), 0)
    # wheel of 199 ring edges and 199 spokes, minus 41 ring edges and 28 spokes
    assert int((L < 0).sum() // 2) == 398 - 41 - 28
    # the graph stays connected: one zero eigenvalue
    assert (np.linalg.eigvalsh(L) < 1e-9).sum() == 1
    A, C = agent_network(L)
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).max() < 0
    # coupling block B K C = [[0.5, -0.1], [-0.1, 0.5]] between neighbours
    i, j = np.argwhere(L == -1)[0]
    assert np.allclose(A[2 * i:2 * i + 2, 2 * j:2 * j + 2], [[0.5, -0.1], [-0.1, 0.5]])
    p = ex3_problem(200, 41)
    v = np.array([1.5, 1.5, -2.0, -2.0])
    D = p.A0 - (p.U * v) @ p.V.T
    # only the off-diagonal entries of agents 21 and 22's diagonal blocks change
    diff = D - p.A0
    assert np.count_nonzero(diff) == 4
    assert diff[40, 41] == diff[41, 40] == -1.5 and diff[42, 43] == diff[43, 42] == 2.0


def test_stability_filter_agrees_with_eigenvalues():
    rng = np.random.default_rng(5)
    grid = ex3_grid()
    for k in (41, 121):
        p = ex3_problem(200, k)
        mask = stable_mask(p, grid)
        # every unstable point and as many stable ones, by brute force
        idx = np.concatenate([np.nonzero(~mask)[0][:40], rng.choice(np.nonzero(mask)[0], 40, replace=False)])
        for i in idx:
            lam = np.linalg.eigvals(p.A0 - (p.U * grid[i]) @ p.V.T).real.max()
            assert (lam < 0) == mask[i]


def test_rayleigh_generator_is_the_physical_linearisation():
    rng = np.random.default_rng(11)
    m = 7
    springs = rng.uniform(0.5, 2.0, m + 1)
    masses = rng.uniform(1.0, 3.0, m)
    a, b = 0.05, 0.01
    p = rayleigh_chain(springs, masses, a, b, [2, 6])
    K = p.meta["K"]
    M = np.diag(masses)
    B = np.zeros((m, 2))
    B[1, 0] = B[5, 1] = 1.0
    v = np.array([0.7, 3.0])
    Cv = a * M + b * K + B @ np.diag(v) @ B.T
    Ap = np.block([[np.zeros((m, m)), np.eye(m)], [-np.linalg.solve(M, K), -np.linalg.solve(M, Cv)]])
    # the API's A(v) = A0 - U diag(v) V^T is the transpose of the paper's A_p(v)
    assert np.allclose((p.A0 - (p.U * v) @ p.V.T).T, Ap)
    Z = np.block([[np.linalg.inv(K), np.zeros((m, m))], [np.zeros((m, m)), np.linalg.inv(M)]])
    assert np.allclose(p.G @ p.G.T, Z)
    # seed solution: trace of the corrected closed form (§3.1)
    X0 = ol.lyap_solve(p.A0, p.G @ p.G.T)
    Ki = np.linalg.inv(K)
    X11 = np.linalg.inv(a * K + b * K @ np.linalg.solve(M, K)) + 0.5 * a * Ki @ M @ Ki + 0.5 * b * Ki
    X22 = np.linalg.inv(a * M + b * K)
    assert abs(np.trace(X0) - (np.trace(X11) + np.trace(X22))) <= 1e-12 * np.trace(X0)
    # and the oracle's f at a small v approaches it
    f = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, np.array([1e-9, 1e-9]))
    assert abs(f - np.trace(X0)) <= 1e-6 * np.trace(X0)
