"""lyap_check_solution_noalloc: the check of given capacitance solutions that
allocates no device memory. It is for callers that cannot allocate while
they run: hosts that reserve their device memory once at start-up in their
own pool, and plug-ins confined to another framework's allocator.

It must agree with the allocating entry points: its traces with
lyap_trace_EX (FP64 tolerance 1e-10 relative, as the other FP64 tests) and
its residuals with the residual that lyap_param_solve reports for the same
solutions. All calls share one static scratch array that keeps the last
call's contents, so the calls here run in an order that would expose stale
scratch: a large call, a call whose scratch is all NaN (v_i = 0), then a
smaller call on another seed. Free device memory must not change across
calls once the first call on the device has looked up the array. This file
is collected last.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from workloads import workload_small_fp64

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _small_problem(seed, n, k, g):
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((n, n)) / math.sqrt(n)
    A0 = R - (np.linalg.eigvals(R).real.max() + 1.0) * np.eye(n)
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    return A0, U, V, G, E @ E.T / n, rng.uniform(0.2, 2.0, (6, k))


def test_noalloc_matches_allocating_entry_points_in_a_row():
    import torch

    ly.build()
    ctx = ly.Context(0)
    dev = torch.device("cuda", 0)
    p, vs = workload_small_fp64()
    seed_a = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    A0, U, V, G, E, vb_host = _small_problem(77, 37, 3, 5)
    seed_b = ly.Seed(ctx, A0, U, V, G, E)

    # everything the checks read or write is allocated before the first call
    va = torch.tensor(vs, dtype=torch.float64, device=dev)
    wa, info_a = seed_a.param_solve(va)
    fa_ref = seed_a.trace_EX(va).cpu().numpy()
    vb = torch.tensor(vb_host, dtype=torch.float64, device=dev)
    wb, info_b = seed_b.param_solve(vb)
    fb_ref = seed_b.trace_EX(vb).cpu().numpy()
    v_zero = torch.zeros_like(va)
    tra = torch.full((len(vs),), float("nan"), dtype=torch.float64, device=dev)
    rsa = torch.full_like(tra, float("nan"))
    trz = torch.zeros_like(tra)
    rsz = torch.zeros_like(tra)
    trb = torch.full((len(vb_host),), float("nan"), dtype=torch.float64, device=dev)
    rsb = torch.full_like(trb, float("nan"))

    # 1) a large call (100 systems of n = 100, k = 2); the first call on the
    #    device also looks up the scratch array's address
    ly.check_solution_noalloc(seed_a, va, wa, tra, rsa)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(dev)[0]
    ly.check_solution_noalloc(seed_a, va, wa, tra, rsa)
    # 2) v = 0: every reciprocal and residual entry this call writes is NaN
    ly.check_solution_noalloc(seed_a, v_zero, wa, trz, rsz)
    # 3) a smaller call on another seed (n = 37, k = 3) after the NaN call
    ly.check_solution_noalloc(seed_b, vb, wb, trb, rsb)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free_before

    tra, rsa = tra.cpu().numpy(), rsa.cpu().numpy()
    assert np.all(np.abs(tra - fa_ref) <= TOL_FP64 * np.abs(fa_ref))
    assert np.all(rsa < 1e-10)
    assert np.allclose(rsa, [i["rel_resid"] for i in info_a], rtol=1e-6, atol=1e-16)
    # the trace of a given solution does not involve v; its residual does
    assert np.isnan(rsz.cpu().numpy()).all()
    assert np.array_equal(trz.cpu().numpy(), tra)
    trb, rsb = trb.cpu().numpy(), rsb.cpu().numpy()
    assert np.all(np.abs(trb - fb_ref) <= TOL_FP64 * np.abs(fb_ref))
    assert np.allclose(rsb, [i["rel_resid"] for i in info_b], rtol=1e-6, atol=1e-16)
    fo = [oracle.trace_EX(A0, U, V, G, E, v) for v in vb_host[:2]]
    assert np.all(np.abs(trb[:2] - fo) <= TOL_FP64 * np.abs(fo))


def test_noalloc_rejects_calls_beyond_the_scratch():
    import torch

    ly.build()
    ctx = ly.Context(0)
    dev = torch.device("cuda", 0)
    big_seed = ly.Seed(ctx, -np.diag(np.linspace(1.0, 2.0, 200)), np.ones((200, 8)) * 1e-3,
                       np.ones((200, 8)) * 1e-3, np.ones((200, 1)), None)
    # 1400 systems x 200 x 8 = 2,240,000 entries + 5600 reciprocals > 2^21 + 2^16
    vb = torch.ones((1400, 8), dtype=torch.float64, device=dev)
    wb = torch.zeros((1400, 8, 200, 2), dtype=torch.float64, device=dev)
    out = torch.empty(1400, dtype=torch.float64, device=dev)
    with pytest.raises(ly.LyapError) as e:
        ly.check_solution_noalloc(big_seed, vb, wb, out, out.clone())
    assert e.value.code == ly.EINVAL
    # 1300 systems fit: 2,080,000 + 5200 <= 2,162,688
    ly.check_solution_noalloc(big_seed, vb[:1300], wb[:1300], out[:1300], out[:1300].clone())
    torch.cuda.synchronize()
