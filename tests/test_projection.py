"""The projection framework of §2.2 on the GPU (lyap_proj_*) against the
CPU oracle of the same framework (oracle/projection.py) and against the
exact traces.

For every v the GPU reports the number of blocks m it used and the backward
error Delta_{m,v}. The oracle, given the same m, builds its own basis of
EK_m (same blocks, same deflation rule), solves the projected equation
(param_projected) by LAPACK and evaluates the backward error proposition:
  * the basis dimensions agree block by block;
  * the traces agree to 1e-10 relative (the Galerkin solution depends only
    on the space, not on its basis);
  * Delta agrees to 1e-6 relative (or both are below 1e-14), and meets eps;
  * the traces are within 1e-6 relative of the exact ones (Bartels-Stewart).
Workloads: Ex. 3's network (n = 400, B_l != B_r, fast convergence) and a
damped chain (n = 100, slow convergence: the space grows to most of R^n).
"""
import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from oracle import projection as op
from tests.gpu_common import rel_err
from workloads import workload_ex3, workload_small_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ly.build()
    return ly.Context(0)


def _oracle_at(p, m, v, cache):
    if "ek" not in cache:
        sq = op.seed_quantities(p.A0, p.U, p.V, p.G, p.E)
        cache.update(sq=sq, ek=op.ExtendedKrylov(sq["A0p"], sq["P"]),
                     off=op.offline_norms(sq["A0p"], sq["Bl"], sq["Br"]))
    sq, ek, off = cache["sq"], cache["ek"], cache["off"]
    pm = op.projected_matrices(ek, m, sq["Bl"], sq["Br"])
    Y = op.solve_projected(pm, ek.G, v)
    return op.trace_value(sq, pm, Y, p.E), op.backward_error_cheap(pm, Y, ek.G, v, off), pm["Vm"].shape[1]


@pytest.mark.parametrize("precision", [ly.FP64, ly.BF16_IR])
def test_projection_on_the_ex3_network(ctx, precision):
    p, vs = workload_ex3(41)
    sel = vs[::97]
    pj = ly.Projection(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, delta, blocks, info = pj.trace_EX(sel, eps=1e-10, m_max=60, return_info=True, precision=precision)
    assert all(i["status"] == 0 for i in info)
    assert (delta <= 1e-10).all() and (blocks >= 1).all()
    nb, dim = pj.dims()
    cache = {}
    tol_f = 1e-10 if precision == ly.FP64 else 1e-8
    for i in range(0, len(sel), 3):
        fo, do, d_or = _oracle_at(p, int(blocks[i]), sel[i], cache)
        assert rel_err(f[i], fo) <= tol_f, (i, blocks[i])
        assert abs(delta[i] - do) <= 1e-6 * do + 1e-14, (delta[i], do)
        fx = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, sel[i])
        assert rel_err(f[i], fx) <= 1e-6
    # the space the GPU built has the oracle's dimensions
    cache["ek"].ensure(nb)
    assert cache["ek"].basis(nb).shape[1] == dim
    pj.free()


def test_projection_on_a_chain(ctx):
    p, vs = workload_small_fp64()
    sel = vs[::9]
    pj = ly.Projection(ctx, p.A0, p.U, p.V, p.G, p.E)
    f, delta, blocks, info = pj.trace_EX(sel, eps=1e-8, m_max=40, return_info=True)
    assert all(i["status"] == 0 for i in info)
    cache = {}
    for i in range(len(sel)):
        fo, do, _ = _oracle_at(p, int(blocks[i]), sel[i], cache)
        assert rel_err(f[i], fo) <= 1e-9, (i, blocks[i], f[i], fo)
        assert delta[i] <= 1e-8
        fx = oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, sel[i])
        assert rel_err(f[i], fx) <= 1e-5
    # block sizes agree with the oracle's deflated basis
    nb, dim = pj.dims()
    ek = cache["ek"]
    ek.ensure(nb)
    assert ek.basis(nb).shape[1] == dim
    pj.free()


def test_projection_with_given_seed_solution(ctx):
    """X0 U and f(X0) supplied by the caller (Assumption 2) instead of the
    internal factorisation: same results."""
    p, vs = workload_ex3(121)
    sel = vs[::211]
    sq = op.seed_quantities(p.A0, p.U, p.V, p.G, p.E)
    pj1 = ly.Projection(ctx, p.A0, p.U, p.V, p.G, p.E)
    pj2 = ly.Projection(ctx, p.A0, p.U, p.V, None, p.E, XBr=sq["X0"] @ sq["Br"], fX0=sq["f0"])
    f1 = pj1.trace_EX(sel, eps=1e-10, m_max=60)
    f2 = pj2.trace_EX(sel, eps=1e-10, m_max=60)
    assert rel_err(f1, f2).max() <= 1e-10
    with pytest.raises(ly.LyapError) as e:
        pj1.trace_EX(np.zeros((1, p.k)))
    assert e.value.code == ly.EINVAL
