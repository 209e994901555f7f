"""The torch.autograd.Function around the adjoint gradient, and the device
(stream-ordered) path of the C ABI.

TraceEX.apply(v, seed, opts) returns f(v) = trace(E X(v)); backward returns
grad_out[:, None] * df/dv from the library's adjoint capacitance solve
(transpose of eq. (SMW_linearsystem)). Checked element by element against
the oracle's adjoint-Lyapunov gradient and against central differences of
the GPU traces, for CUDA and CPU inputs, FP64 and the mixed path.
Tolerances: traces 1e-10 (FP64) / 1e-8 (mixed) relative; gradients 1e-8
(FP64) / 1e-6 (mixed) relative to the largest component; central
differences (h = 1e-6 v_i) 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2312_08201_gb300 as ly
from tests.gpu_common import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    ly.build()
    ctx = ly.Context(0)
    rng = np.random.default_rng(2024)
    n, k, g = 37, 3, 5
    R = rng.standard_normal((n, n)) / math.sqrt(n)
    A0 = R - (np.linalg.eigvals(R).real.max() + 1.0) * np.eye(n)
    U = rng.standard_normal((n, k)) * 0.3
    V = rng.standard_normal((n, k)) * 0.3
    G = rng.standard_normal((n, g))
    E = rng.standard_normal((n, n))
    E = E @ E.T / n
    vs = rng.uniform(0.2, 2.0, (4, k))
    seed = ly.Seed(ctx, A0, U, V, G, E)
    ref = [oracle.gradient(A0, U, V, G, E, v) for v in vs]
    return ctx, seed, vs, ref, (A0, U, V, G, E)


@pytest.mark.parametrize("device", ["cuda", "cpu"])
@pytest.mark.parametrize("precision,tf,tg", [(ly.FP64, 1e-10, 1e-8), (ly.BF16_IR, 1e-8, 1e-6)])
def test_trace_ex_function_gradient(problem, device, precision, tf, tg):
    import torch

    ctx, seed, vs, ref, mats = problem
    TraceEX = ly.trace_ex_function()
    v = torch.tensor(vs, dtype=torch.float64, device=device, requires_grad=True)
    f = TraceEX.apply(v, seed, {"precision": precision})
    assert f.device == v.device and f.dtype == torch.float64 and f.shape == (len(vs),)
    wts = torch.tensor([1.0, 2.0, -1.0, 0.5], dtype=torch.float64, device=device)
    (f * wts).sum().backward()
    assert v.grad.device == v.device and v.grad.dtype == v.dtype
    fh = f.detach().cpu().numpy()
    gh = v.grad.cpu().numpy()
    for i, (fo, go) in enumerate(ref):
        assert rel_err(fh[i], fo) <= tf
        assert np.abs(gh[i] - wts[i].item() * go).max() <= tg * abs(wts[i].item()) * np.abs(go).max()
    # central differences of the GPU's own FP64 traces
    x = vs[1]
    for j in range(seed.k):
        h = 1e-6 * x[j]
        vp, vm = x.copy(), x.copy()
        vp[j] += h
        vm[j] -= h
        fp, fm = seed.trace_EX(np.stack([vp, vm]), precision=ly.FP64)
        fd = (fp - fm) / (2 * h)
        assert abs(gh[1, j] / 2.0 - fd) <= 1e-5 * max(abs(fd), 1e-6 * abs(fh[1]))


def test_trace_ex_function_float32_input_and_no_grad(problem):
    import torch

    ctx, seed, vs, ref, mats = problem
    TraceEX = ly.trace_ex_function()
    v32 = torch.tensor(vs, dtype=torch.float32, device="cuda", requires_grad=True)
    f = TraceEX.apply(v32, seed)
    f.sum().backward()
    assert v32.grad.dtype == torch.float32
    v_used = v32.detach().double().cpu().numpy()  # the rounded parameters the library solved for
    for i in range(len(vs)):
        fo, go = oracle.gradient(*mats, v_used[i])
        assert rel_err(f[i].item(), fo) <= 1e-10
        assert np.abs(v32.grad[i].double().cpu().numpy() - go).max() <= 1e-6 * np.abs(go).max()
    with torch.no_grad():
        f2 = TraceEX.apply(torch.tensor(vs, device="cuda"), seed)
    assert not f2.requires_grad
    assert rel_err(f2.cpu().numpy(), np.array([r[0] for r in ref])).max() <= 1e-10


@pytest.mark.parametrize("precision,tol", [(ly.FP64, 1e-10), (ly.BF16_IR, 1e-8)])
def test_device_inputs_on_a_side_stream(problem, precision, tol):
    """Device v, device outputs, work queued on a user stream: results match
    the oracle, and the device outputs are written in that stream's order."""
    import torch

    ctx, seed, vs, ref, mats = problem
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        v = torch.tensor(vs, dtype=torch.float64, device="cuda")
        f, g = seed.grad(v, precision=precision)
        f2 = seed.trace_EX(v, precision=precision)
        done = f + 0.0  # queued on s after the call's writes
    s.synchronize()
    assert f.is_cuda and g.is_cuda
    fo = np.array([r[0] for r in ref])
    assert rel_err(done.cpu().numpy(), fo).max() <= tol
    assert rel_err(f2.cpu().numpy(), fo).max() <= tol
    for i, (_, go) in enumerate(ref):
        assert np.abs(g[i].cpu().numpy() - go).max() <= (1e-8 if precision == ly.FP64 else 1e-6) * np.abs(go).max()


def test_device_input_zero_parameter_is_rejected(problem):
    import torch

    ctx, seed, vs, ref, mats = problem
    v = torch.tensor(vs, dtype=torch.float64, device="cuda")
    v[2, 1] = 0.0  # v_i = 0 is excluded (§1); found by the device-side check
    with pytest.raises(ly.LyapError) as e:
        seed.trace_EX(v)
    assert e.value.code == ly.EINVAL
    v[2, 1] = float("inf")
    with pytest.raises(ly.LyapError) as e:
        seed.trace_EX(v, precision=ly.BF16_IR)
    assert e.value.code == ly.EINVAL
    # the seed stays usable
    f = seed.trace_EX(torch.tensor(vs, device="cuda"))
    assert rel_err(f.cpu().numpy(), np.array([r[0] for r in ref])).max() <= 1e-10
