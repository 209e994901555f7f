"""Serving loop: continuous batching across seeds and within a seed,
admission by device memory, latency, and the identity of each result alone
and in the mix.

Alone vs mixed: the same request solved through a server with no other
traffic and inside a concurrent mix of requests on several seeds must agree
to the path's tolerance (1e-8 relative for the mixed path, 1e-10 for FP64):
batching changes the recycled space and the iteration counts, not the
answer. A few results are also checked against the CPU oracle.
"""

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from workloads import mass_spring_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ly.build()
    ctx = ly.Context(0)
    rng = np.random.default_rng(42)
    probs = [
        mass_spring_chain(np.ones(51), 0.04, [10, 35]),
        mass_spring_chain(rng.uniform(0.5, 2.0, 81), 0.04, [5, 40, 77]),
        mass_spring_chain(np.ones(61), 0.04, [3, 20, 33, 58]),
    ]
    seeds = [ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E) for p in probs]
    reqs = []
    for i in range(9):
        si = i % 3
        k = probs[si].k
        reqs.append((si, np.exp(rng.uniform(np.log(0.1), np.log(10.0), (16, k))), i % 4 == 0))
    return ctx, probs, seeds, reqs


def run_requests(ctx, seeds, reqs, precision, **opts):
    srv = ly.Server(ctx, precision=precision, **opts)
    ids = [srv.register(s) for s in seeds]
    tickets = [srv.submit(ids[si], v, g) for si, v, g in reqs]
    srv.run()
    out = [srv.poll(t, len(v), v.shape[1], g) for t, (si, v, g) in zip(tickets, reqs)]
    srv.close()
    return out


@pytest.mark.parametrize("precision,tol", [(ly.BF16_IR, 1e-8), (ly.FP64, 1e-10)])
def test_results_same_alone_and_in_mix(setup, precision, tol):
    ctx, probs, seeds, reqs = setup
    mixed = run_requests(ctx, seeds, reqs, precision)
    for j in (0, 4, 7):
        alone = run_requests(ctx, seeds, [reqs[j]], precision)[0]
        assert np.all(np.abs(mixed[j]["f"] - alone["f"]) <= tol * np.abs(alone["f"]))
        if reqs[j][2]:
            assert np.abs(mixed[j]["g"] - alone["g"]).max() <= 1e-6 * np.abs(alone["g"]).max()
    for r in mixed:
        assert r["latency_s"] > 0
        assert all(i["status"] == 0 for i in r["info"])
    si, v, g = reqs[1]
    p = probs[si]
    ref = [oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, x) for x in v[:3]]
    assert np.all(np.abs(mixed[1]["f"][:3] - ref) <= tol * np.abs(ref))


def test_admission_by_memory_budget(setup):
    ctx, probs, seeds, reqs = setup
    # a budget that holds the seeds and only about one request at a time
    tiny = sum(s.stats()["resident_bytes"] for s in seeds) + 64 << 20
    out = run_requests(ctx, seeds, reqs[:5], ly.BF16_IR, hbm_budget=tiny)
    assert all(r is not None and all(i["status"] == 0 for i in r["info"]) for r in out)
    srv = ly.Server(ctx, hbm_budget=sum(s.stats()["resident_bytes"] for s in seeds) + (1 << 20))
    sid = srv.register(seeds[0])
    with pytest.raises(ly.LyapError) as e:
        srv.submit(sid, np.ones((4000, 2)))
    assert e.value.code == ly.ENOMEM
    srv.close()


def test_cancel_and_bad_input(setup):
    ctx, probs, seeds, reqs = setup
    # room for one 16-vector request but not two
    probe = ly.Server(ctx)
    one = probe.estimate(probe.register(seeds[1]), 16)
    probe.close()
    srv = ly.Server(ctx, hbm_budget=sum(s.stats()["resident_bytes"] for s in seeds) + one + one // 2)
    sid = srv.register(seeds[1])
    t1 = srv.submit(sid, reqs[1][1])
    t2 = srv.submit(sid, reqs[1][1])
    t3 = srv.submit(sid, reqs[1][1])
    srv.cancel(t3)  # queued behind the budget: cancellable (or already admitted: completes)
    srv.run()
    assert srv.poll(t1, 16, 3) is not None
    assert srv.poll(t2, 16, 3) is not None
    bad = reqs[1][1].copy()
    bad[0, 0] = 0.0
    with pytest.raises(ly.LyapError):
        srv.submit(sid, bad)
    srv.close()


def test_request_for_a_busy_seed_overtakes_a_long_request(setup):
    """Mixed-precision traces join a seed's running set at the next
    refinement step: a short request submitted while a long one occupies the
    seed finishes first, and its results equal those of the same request
    alone (1e-8) and the oracle's."""
    import time

    ctx, probs, seeds, reqs = setup
    rng = np.random.default_rng(9)
    k = probs[0].k
    long_v = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (1536, k)))
    short_v = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (8, k)))
    srv = ly.Server(ctx, precision=ly.BF16_IR, batch=128)
    sid = srv.register(seeds[0])
    t_long = srv.submit(sid, long_v)
    time.sleep(0.05)
    t_short = srv.submit(sid, short_v)
    done = {}
    while len(done) < 2:
        for name, t, nv in (("long", t_long, len(long_v)), ("short", t_short, len(short_v))):
            if name not in done:
                r = srv.poll(t, nv, k)
                if r is not None:
                    done[name] = (time.perf_counter(), r)
        time.sleep(0.002)
    srv.close()
    assert done["short"][0] < done["long"][0]
    assert done["short"][1]["latency_s"] < done["long"][1]["latency_s"]
    alone = run_requests(ctx, seeds, [(0, short_v, False)], ly.BF16_IR)[0]
    fs = done["short"][1]["f"]
    assert np.all(np.abs(fs - alone["f"]) <= 1e-8 * np.abs(alone["f"]))
    p = probs[0]
    ref = [oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, x) for x in short_v[:2]]
    assert np.all(np.abs(fs[:2] - ref) <= 1e-8 * np.abs(ref))
    fl = done["long"][1]["f"]
    ref = [oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, x) for x in long_v[[0, 1535]]]
    assert np.all(np.abs(fl[[0, 1535]] - ref) <= 1e-8 * np.abs(ref))
    assert all(i["status"] == 0 for i in done["long"][1]["info"])
