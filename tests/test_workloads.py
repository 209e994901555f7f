"""Full-size workloads in the configuration the library runs them:
  * differentiation: 1000-mass chain (n = 2000), 4 dampers, E = projector on
    the first 100 modal displacements, 256 parameter vectors with gradients;
  * multi-agent: 256 agents (n = 1024), 8 tunable edges, 512 weight vectors
    solved as one lockstep batch;
  * serving: two 400-mass seeds of the serving workload through the server.
Outputs are sampled against the oracle (one solve at n = 2000 costs about
half a minute of CPU: gradients at the first and last vector, the trace at
a middle one), the rest against the FP64 GPU path and against central
differences.
Tolerances: 1e-10 (FP64 traces), 1e-8 (mixed traces), gradients 1e-8
(FP64) / 1e-6 (mixed) relative to the largest component, central
differences 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err
from workloads import workload_differentiation, workload_multi_agent, workload_serving_seeds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ly.build()
    return ly.Context(0)


def test_differentiation_workload_full_size(ctx):
    p, vs = workload_differentiation()  # Haar-dense
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    f16, g16, i16 = seed.grad(vs, return_info=True, precision=ly.BF16_IR)
    f64, g64, i64 = seed.grad(vs, return_info=True, precision=ly.FP64)
    assert all(i["status"] == 0 for i in i16) and all(i["status"] == 0 for i in i64)
    assert rel_err(f16, f64).max() <= 1e-8
    scale = np.abs(g64).max(axis=1)
    assert (np.abs(g16 - g64).max(axis=1) <= 1e-6 * scale).all()
    # the oracle on the structured problem (f and its gradient are invariant
    # under the orthogonal similarity)
    # at the first, a middle and the last of the 256 vectors
    ps, _ = workload_differentiation(dense=False)
    for i in (0, len(vs) - 1):
        fo, go = oracle.gradient(ps.A0, ps.U, ps.V, ps.G, ps.E, vs[i])
        assert rel_err(f64[i], fo) <= 1e-10, i
        assert rel_err(f16[i], fo) <= 1e-8, i
        assert np.abs(g64[i] - go).max() <= 1e-8 * np.abs(go).max(), i
        assert np.abs(g16[i] - go).max() <= 1e-6 * np.abs(go).max(), i
    i = len(vs) // 2
    fo = oracle.trace_EX(ps.A0, ps.U, ps.V, ps.G, ps.E, vs[i])
    assert rel_err(f64[i], fo) <= 1e-10
    assert rel_err(f16[i], fo) <= 1e-8
    # central differences of GPU traces
    v = vs[1]
    for j in range(p.k):
        h = 1e-6 * v[j]
        vp, vm = v.copy(), v.copy()
        vp[j] += h
        vm[j] -= h
        fp, fm = seed.trace_EX(np.stack([vp, vm]), precision=ly.FP64)
        fd = (fp - fm) / (2 * h)
        assert abs(g64[1, j] - fd) <= 1e-5 * max(abs(fd), 1e-6 * abs(f64[1]))


def test_multi_agent_workload_one_batch(ctx):
    p, ws = workload_multi_agent()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    st = seed.stats()
    assert st["real_path"] == 1  # symmetric A0: real eigenvalues
    f16, info = seed.trace_EX(ws, return_info=True, precision=ly.BF16_IR, batch=len(ws))
    f64 = seed.trace_EX(ws, precision=ly.FP64, batch=len(ws))
    assert all(i["status"] == 0 for i in info)
    assert rel_err(f16, f64).max() <= 1e-8
    for i in (0, 511):
        fo = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, ws[i])
        assert rel_err(f64[i], fo) <= 1e-10
        assert rel_err(f16[i], fo) <= 1e-8


def test_serving_workload_seeds_through_server(ctx):
    probs = workload_serving_seeds(dense=True, sizes=(400,))
    seeds = [ly.Seed(ctx, q.A0, q.U, q.V, q.G, q.E) for q in probs]
    rng = np.random.default_rng(3)
    srv = ly.Server(ctx, precision=ly.BF16_IR)
    ids = [srv.register(s) for s in seeds]
    reqs = [(i % 2, np.exp(rng.uniform(np.log(0.1), np.log(10.0), (64, probs[i % 2].k)))) for i in range(4)]
    tickets = [srv.submit(ids[si], v) for si, v in reqs]
    srv.run()
    outs = [srv.poll(t, 64, v.shape[1]) for t, (si, v) in zip(tickets, reqs)]
    srv.close()
    for (si, v), r in zip(reqs[:2], outs[:2]):
        q = probs[si]
        fo = oracle.trace_EX(q.A0, q.U, q.V, q.G, q.E, v[5])
        assert rel_err(r["f"][5], fo) <= 1e-8
        assert all(i["status"] == 0 for i in r["info"])


def test_serving_seed_of_3200_states_against_the_oracle(ctx):
    """The largest serving seed (1600 masses, n = 3200) through the server's
    engine: its refinement residual runs the integer-sliced product in four
    K chunks (2n = 6400). One parameter vector against the oracle (about two
    minutes of CPU), the request's others against the FP64 GPU path."""
    probs = workload_serving_seeds(dense=True, sizes=(1600,))
    structured = workload_serving_seeds(dense=False, sizes=(1600,))[0]  # the same first seed, unrotated
    q = probs[0]
    assert q.n == 3200 and structured.k == q.k
    seed = ly.Seed(ctx, q.A0, q.U, q.V, q.G, q.E)
    rng = np.random.default_rng(17)
    v = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (16, q.k)))
    srv = ly.Server(ctx, precision=ly.BF16_IR)
    sid = srv.register(seed)
    t = srv.submit(sid, v)
    srv.run()
    r = srv.poll(t, 16, q.k)
    srv.close()
    assert all(i["status"] == 0 for i in r["info"])
    f64 = seed.trace_EX(v[:3], precision=ly.FP64)
    assert rel_err(r["f"][:3], f64).max() <= 1e-8
    fo = oracle.trace_EX(structured.A0, structured.U, structured.V, structured.G, structured.E, v[0])
    assert rel_err(r["f"][0], fo) <= 1e-8
    assert rel_err(f64[0], fo) <= 1e-10
