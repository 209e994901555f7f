"""lyap_check_solution_noalloc: the allocation-free check of given
capacitance solutions, for callers that may not allocate device memory
(graph capture, fixed start-up pools, host-framework allocators).

It must agree with the allocating entry points: its traces with
lyap_trace_EX (FP64 tolerance 1e-10 relative, as the other FP64 tests) and
its residuals with the residual that lyap_param_solve reports for the same
solutions. Two calls in a row share the static scratch array; the second
must not see the first's leftovers. This file is collected last.
"""
import numpy as np
import pytest

import paper_2312_08201_gb300 as ly
from workloads import workload_small_fp64

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def test_noalloc_matches_allocating_entry_points_twice():
    import torch

    ly.build()
    ctx = ly.Context(0)
    p, vs = workload_small_fp64()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    dev = torch.device("cuda", 0)
    for lo, hi in ((0, 40), (40, 100)):  # two calls in a row with different sizes
        v = torch.tensor(vs[lo:hi], dtype=torch.float64, device=dev)
        w, info = seed.param_solve(v)
        f_ref = seed.trace_EX(v).cpu().numpy()
        tr = torch.full((hi - lo,), float("nan"), dtype=torch.float64, device=dev)
        rs = torch.full((hi - lo,), float("nan"), dtype=torch.float64, device=dev)
        ly.check_solution_noalloc(seed, v, w, tr, rs)
        torch.cuda.synchronize()
        tr = tr.cpu().numpy()
        rs = rs.cpu().numpy()
        assert np.all(np.abs(tr - f_ref) <= TOL_FP64 * np.abs(f_ref))
        rel_ref = np.array([i["rel_resid"] for i in info])
        assert np.all(rs < 1e-10)
        assert np.allclose(rs, rel_ref, rtol=1e-6, atol=1e-16)
    too_many = torch.ones((1400, 2), dtype=torch.float64, device=dev)
    wbig = torch.zeros((1400, 2, 100, 2), dtype=torch.float64, device=dev)
    out = torch.empty(1400, dtype=torch.float64, device=dev)
    ok = ly.check_solution_noalloc(seed, too_many[:10], wbig[:10], out[:10], out[:10].clone())
    assert ok is None
    big_seed = ly.Seed(ctx, np.kron(np.eye(20), p.A0[:10, :10] * 0 - np.eye(10)), np.ones((200, 8)) * 1e-3,
                       np.ones((200, 8)) * 1e-3, np.ones((200, 1)), None)
    vb = torch.ones((1400, 8), dtype=torch.float64, device=dev)
    wb = torch.zeros((1400, 8, 200, 2), dtype=torch.float64, device=dev)
    with pytest.raises(ly.LyapError) as e:
        ly.check_solution_noalloc(big_seed, vb, wb, out, out.clone())
    assert e.value.code == ly.EINVAL
