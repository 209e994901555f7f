"""Benchmark: trace(E X(v)) evaluations per second on one GB300.

A step is one pass of the hot path over the 800-state damped chain
(400 unit masses, 401 springs U[0.5, 2], alpha = 0.04, two dampers at
random masses, seeded Haar similarity so the solver sees dense data) for
1000 parameter pairs drawn log-uniformly on [1e-2, 1e2]^2 and ordered along
a nearest-neighbour path: the seed stays factored on the device, and each
step evaluates f(v) = trace(E X(v)) for all 1000 v through the library
(capacitance solves, refinement, trace epilogue).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--precision best|fp64|bf16_ir]
Prints one JSON line (rank 0). Multi-GPU runs are independent replicas
(weak scaling): each rank sweeps its own copy of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trace(EX(v)) evals/sec at rel err<=1e-8 vs FP64 path; p50/p99 request latency"
WORKLOAD = "chain400 n=800 k=2, 1000 v log-uniform [1e-2,1e2]^2 NN-ordered, Haar-dense"
FP64_PEAK_FLOPS_PER_CLK_SM = 4.0  # 2 FP64 FMA per clock per SM (1.25 TFLOP/s at 2070 MHz x 152 SMs)
SMS = 152
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel,
# averaged over every launch of that kernel in one 1000-vector sweep of this
# workload, from a one-kernel ncu capture (profiles/ortho_cl_800state_1000v.md).
# Valid for the kernel as it stands; a change to the kernel invalidates it.
MEASURED_TRAFFIC_PER_LAUNCH = {"ortho": 106.95e6}
FP32_LANES_PER_SM = 128.0  # FP32 lane-instructions per clock per SM
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["best", "fp64", "bf16_ir"], default="best")
    ap.add_argument("--batch", type=int, default=0, help="systems solved in lockstep (0: library default)")
    ap.add_argument("--pbar", type=int, default=-1, help="TSVD rank of the preconditioner coupling (-1: library default)")
    ap.add_argument("--residual", choices=["ff", "fp64", "tc"], default="tc",
                    help="arithmetic of the mixed path's refinement residual")
    ap.add_argument("--nv", type=int, default=0, help="parameter vectors of the sweep (0: all 1000)")
    ap.add_argument("--s", type=int, default=-1, help="recycled vectors (-1: library default)")
    ap.add_argument("--profile-sweep", action="store_true",
                    help="after the measurements, run one more sweep between cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--cpu-sample", type=int, default=8, help="oracle evaluations in the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["precision", "serving", "kernels"], default="precision")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests per arrival rate")
    ap.add_argument("--serving-sizes", default="200,400,800,1600", help="serving: chain lengths (masses)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-path, gradient, multi-agent and serving figures of the default run")
    ap.add_argument("--serving-requests", type=int, default=160,
                    help="requests of the serving figure in the default run (one rate, 0.95 of saturation)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        loaded = [r["sm"] for r in rows if r["power"] > 200] or [r["sm"] for r in rows]
        return dict(sm_mhz=statistics.median(loaded), sm_max_mhz=max(r["smax"] for r in rows),
                    reasons=sorted(reasons), samples=len(rows), power_w_max=max(r["power"] for r in rows))


# ---------------------------------------------------------------- baseline
CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from workloads import workload_precision
p, vs = workload_precision()
sample = vs[:{count}]
t = time.perf_counter()
f = [oracle.trace_EX(p.A0, p.U, p.V, p.G, p.E, v) for v in sample]
dt = time.perf_counter() - t
print(json.dumps(dict(evals=len(sample), seconds=dt, f=f)))
"""


def cpu_oracle(count: int):
    """Time the oracle on `count` parameter vectors in a fresh process using
    every host core for BLAS (returns evals/s, cores, traces)."""
    cores = len(os.sched_getaffinity(0))
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(cores)
    r = subprocess.run([sys.executable, "-c", CPU_SNIPPET.format(root=ROOT, count=count)], capture_output=True,
                       text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["evals"] / d["seconds"], cores, d["f"], d["seconds"]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0), "fallback"


# --------------------------------------------------------------- reference
def run_reference(args, rank):
    if rank != 0:
        return
    per_step = 2
    vals = []
    cores = None
    for i in range(args.warmup + args.steps):
        rate, cores, _, secs = cpu_oracle(per_step)
        if i >= args.warmup:
            vals.append(secs)
    total = sum(vals)
    value = per_step * args.steps / total
    line = dict(metric=METRIC, value=value, unit="evals/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * total / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, sample_per_step=per_step),
                cpu_baseline=dict(kind="oracle", value=value, unit="evals/s", cores=cores,
                                  sample=f"first {per_step} parameter pairs of the sweep per step, "
                                         "Bartels-Stewart per v in float64"),
                e2e=dict(value=value, unit="evals/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- serving
def serving_measure(ctx, prec, sizes=(200, 400, 800, 1600), requests=2000, fracs=(0.5, 0.8, 0.95), burst=128):
    """Serving workload: 8 seeds (two chains each of the given lengths,
    k in {2,3,4}, Haar-dense), requests of 64 log-uniform parameter vectors
    on [0.1, 10]^k. Saturation throughput from a burst, then Poisson arrivals
    at the given fractions of it; evals/s and p50/p99 submit-to-result
    latency per rate."""
    import threading

    import numpy as np

    import paper_2312_08201_gb300 as ly
    from workloads import workload_serving_requests, workload_serving_seeds

    probs = workload_serving_seeds(dense=True, sizes=sizes)
    t0 = time.perf_counter()
    seeds = [ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E) for p in probs]
    t_factor = time.perf_counter() - t0

    def drive(reqs, paced):
        srv = ly.Server(ctx, precision=prec)
        ids = [srv.register(sd) for sd in seeds]
        tickets = [None] * len(reqs)
        start = time.perf_counter()

        def submitter():
            for i, (ta, si, v) in enumerate(reqs):
                if paced:
                    delay = start + ta - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets[i] = srv.submit(ids[si], v)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        srv.run()
        elapsed = time.perf_counter() - start
        lat = []
        evals = 0
        for t, (ta, si, v) in zip(tickets, reqs):
            r = srv.poll(t, len(v), v.shape[1])
            lat.append(r["latency_s"])
            evals += len(v)
        srv.close()
        return evals / elapsed, lat

    # warm-up (recycle spaces, workspaces) and saturation
    warm = workload_serving_requests(probs, rate_hz=1e9, count=16, seed=99)
    drive(warm, False)
    sat, _ = drive(workload_serving_requests(probs, rate_hz=1e9, count=min(burst, requests), seed=1), False)
    rates = {}
    for frac in fracs:
        req_rate = frac * sat / 64.0
        reqs = workload_serving_requests(probs, rate_hz=req_rate, count=requests, seed=int(frac * 100))
        thr, lat = drive(reqs, True)
        rates[str(frac)] = dict(evals_per_s=thr, p50_ms=1e3 * float(np.percentile(lat, 50)),
                                p99_ms=1e3 * float(np.percentile(lat, 99)), requests=len(reqs))
    for sd in seeds:
        sd.free()
    return dict(workload=f"8 chain seeds {sizes} masses x2, k in {{2,3,4}}, Haar-dense, 64 v log-uniform "
                         "[0.1,10]^k per request, Poisson arrivals",
                n=[p.n for p in probs], k=[p.k for p in probs], saturation_evals_per_s=sat, rates=rates,
                seed_factor_s=t_factor)


def run_serving(args, local):
    import torch

    import paper_2312_08201_gb300 as ly

    torch.cuda.set_device(local)
    ly.build()
    sizes = tuple(int(x) for x in args.serving_sizes.split(","))
    ctx = ly.Context(local)
    prec = ly.FP64 if args.precision == "fp64" else ly.BF16_IR
    sv = serving_measure(ctx, prec, sizes, args.requests)
    rates = sv["rates"]
    line = dict(metric=METRIC, value=rates["0.95"]["evals_per_s"], unit="evals/s", n_gpus=1, steps=args.requests,
                warmup=16, ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="bf16x3-gemm/f32-krylov/int-sliced-bf16-refine" if prec == ly.BF16_IR
                else "f64", data="synthetic",
                config=dict(workload="serving: " + sv["workload"], n=sv["n"], k=sv["k"]),
                saturation_evals_per_s=sv["saturation_evals_per_s"], rates=rates, seed_factor_s=sv["seed_factor_s"],
                latency_ms=dict(p50=rates["0.95"]["p50_ms"], p99=rates["0.95"]["p99_ms"], request="64-vector sweep"))
    print(json.dumps(line), flush=True)


# ---------------------------------------------- the other workloads (extras)
def _event_time(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    out = None
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ms], out


def extra_fp64_path(seed, v_dev, f64_ref, stream, steps=2):
    """The plain FP64 GPU path on the headline sweep (the path the mixed one
    is compared with)."""
    import numpy as np

    import paper_2312_08201_gb300 as ly

    ms, f = _event_time(lambda: seed.trace_EX(v_dev, precision=ly.FP64), steps, 1, stream)
    f = f.cpu().numpy()
    rep = np.abs(f - f64_ref) / np.abs(f64_ref)
    return dict(evals_per_s=len(f) * len(ms) / (sum(ms) / 1e3), ms_per_sweep=float(np.mean(ms)), steps=len(ms),
                max_rel_diff_between_runs=float(rep.max()), dtype="f64")


def extra_grad(ctx, dev, stream, steps=2):
    """Differentiation workload: 1000-mass chain (n = 2000), 4 dampers,
    E = first 100 modal displacements, 256 v with gradients, mixed path; the
    first 4 v also on the FP64 path for the accuracy figures."""
    import numpy as np
    import torch

    import paper_2312_08201_gb300 as ly
    from workloads import workload_differentiation

    p, vs = workload_differentiation()
    t0 = time.perf_counter()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    tf = time.perf_counter() - t0
    v = torch.tensor(vs, dtype=torch.float64, device=dev)
    ms, (f, g) = _event_time(lambda: seed.grad(v, precision=ly.BF16_IR), steps, 1, stream)
    f64, g64 = seed.grad(v[:4], precision=ly.FP64)
    f, g, f64, g64 = (x.cpu().numpy() for x in (f, g, f64, g64))
    gerr = float(max(np.abs(g[i] - g64[i]).max() / np.abs(g64[i]).max() for i in range(4)))
    seed.free()
    return dict(workload="chain1000 n=2000 k=4, E = first 100 modal displacements, 256 v log-uniform [0.1,10]^4, "
                         "Haar-dense", unit="evals+grads/s", value=len(vs) * len(ms) / (sum(ms) / 1e3),
                ms_per_sweep=float(np.mean(ms)), precision="bf16_ir",
                max_rel_err_f_vs_fp64_path=float(np.max(np.abs(f[:4] - f64) / np.abs(f64))),
                max_rel_err_grad_vs_fp64_path=gerr, seed_factor_s=tf)


def extra_ex3(ctx, dev, stream):
    """Ex. 3 of the paper: the 200-agent network of Algorithm 2, a rank-4
    change with B_l != B_r at the four positions of the example's table,
    the stable members of the 40 x 40 grid (6,044 systems in all, negative
    parameters included). Small-scale path (mixed precision, one batch per
    position) and the projection framework (backward error 1e-10, the
    paper's setting), each timed over the whole sweep; both against the FP64
    small-scale path on the same v."""
    import numpy as np
    import torch

    import paper_2312_08201_gb300 as ly
    from workloads import EX3_POSITIONS, workload_ex3

    probs = [workload_ex3(kp) for kp in EX3_POSITIONS]
    seeds = [ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E) for p, _ in probs]
    vdev = [torch.tensor(vs, dtype=torch.float64, device=dev) for _, vs in probs]
    total = sum(len(vs) for _, vs in probs)
    ref = [sd.trace_EX(v, precision=ly.FP64).cpu().numpy() for sd, v in zip(seeds, vdev)]

    def small():
        return [sd.trace_EX(v, precision=ly.BF16_IR) for sd, v in zip(seeds, vdev)]

    ms, out = _event_time(small, 2, 1, stream)
    err_small = max(float(np.max(np.abs(o.cpu().numpy() - r) / np.abs(r))) for o, r in zip(out, ref))
    for sd in seeds:
        sd.free()
    # projection framework: the space is built once per position (offline,
    # reported separately) and then serves the sweep
    t0 = time.perf_counter()
    projs = [ly.Projection(ctx, p.A0, p.U, p.V, p.G, p.E) for p, _ in probs]
    t_off = time.perf_counter() - t0
    for pj, (p, vs) in zip(projs, probs):
        pj.trace_EX(vs[:8], eps=1e-10, m_max=200)  # warm-up: grows the spaces
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outp = [pj.trace_EX(vs, eps=1e-10, m_max=200, return_info=True) for pj, (p, vs) in zip(projs, probs)]
    t_proj = time.perf_counter() - t0
    err_proj = max(float(np.max(np.abs(o[0] - r) / np.abs(r))) for o, r in zip(outp, ref))
    dims = [pj.dims()[1] for pj in projs]
    blocks = np.concatenate([o[2] for o in outp])
    for pj in projs:
        pj.free()
    return dict(workload="Ex. 3: 200 agents (Algorithm 2 graph), n=400, k=4 (B_l != B_r), positions "
                         f"{list(EX3_POSITIONS)}, {total} stable grid points",
                unit="evals/s",
                small_scale=dict(value=total * len(ms) / (sum(ms) / 1e3), ms_per_sweep=float(np.mean(ms)),
                                 precision="bf16_ir", max_rel_err_vs_fp64_path=err_small),
                projection=dict(value=total / t_proj, s_per_sweep=t_proj, eps=1e-10, offline_s=t_off,
                                basis_dims=dims, blocks_mean=float(blocks.mean()), blocks_max=int(blocks.max()),
                                max_rel_err_vs_fp64_path=err_proj, precision="fp64",
                                timing="wall clock of the host-driven Algorithm 1 (synchronising)"))


def extra_multi_agent(ctx, dev, stream, steps=2):
    """Multi-agent workload: 256 agents (n = 1024), 8 tunable edges, 512
    weight vectors in one lockstep batch, mixed path; 8 of them also on the
    FP64 path."""
    import numpy as np
    import torch

    import paper_2312_08201_gb300 as ly
    from workloads import workload_multi_agent

    p, ws = workload_multi_agent()
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    v = torch.tensor(ws, dtype=torch.float64, device=dev)
    ms, f = _event_time(lambda: seed.trace_EX(v, precision=ly.BF16_IR, batch=len(ws)), steps, 1, stream)
    f64 = seed.trace_EX(v[:8], precision=ly.FP64).cpu().numpy()
    f = f.cpu().numpy()
    st = seed.stats()
    seed.free()
    return dict(workload="256 agents n=1024 k=8 (ER p=0.05), 512 weight vectors U[0.1,5]^8, one batch",
                unit="evals/s", value=len(ws) * len(ms) / (sum(ms) / 1e3), ms_per_sweep=float(np.mean(ms)),
                precision="bf16_ir", real_spectrum=bool(st["real_path"]),
                max_rel_err_vs_fp64_path=float(np.max(np.abs(f[:8] - f64) / np.abs(f64))))


# ------------------------------------------------------------ kernel probe
def run_kernel_probe(args, local):
    """The capacitance operators on a full batch: T(v) applied to 1000
    random inputs of the 800-state seed with the tensor-core operator (panel,
    tcgen05 GEMM, epilogue), the float-float kernel, the integer-sliced
    tensor-core kernel and the FP64 kernel; CUDA-event timing per kernel for
    the roofline, and the errors of the two FP64-accurate operators against
    the FP64 one. One more application of each
    operator runs between cudaProfilerStart/Stop, for ncu captures of full
    launches (--profile-from-start off)."""
    import numpy as np
    import torch

    import paper_2312_08201_gb300 as ly
    from workloads import workload_precision

    torch.cuda.set_device(local)
    ly.build()
    p, vs = workload_precision()
    ctx = ly.Context(local)
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(0)
    v = torch.tensor(vs, dtype=torch.float64, device=dev)
    w = torch.tensor(rng.standard_normal((len(vs), p.k, p.n, 2)), dtype=torch.float64, device=dev)
    for _ in range(2):
        ly.test_apply(seed, v, w, ly.BF16_IR)
        ly.test_apply(seed, v, w, ly.TEST_FF)
        ly.test_apply(seed, v, w, ly.TEST_TC)
        y64 = ly.test_apply(seed, v, w, ly.FP64)
    ly.prof_enable(True)
    for _ in range(max(1, args.steps)):
        ly.test_apply(seed, v, w, ly.BF16_IR)
        yff = ly.test_apply(seed, v, w, ly.TEST_FF)
        ytc = ly.test_apply(seed, v, w, ly.TEST_TC)
    ly.test_apply(seed, v, w, ly.FP64)
    prof, launches = ly.prof_read()
    ly.prof_enable(False)

    def rel(y):
        return float(((y - y64).flatten(1).norm(dim=1) / y64.flatten(1).norm(dim=1)).max())

    ff_err, tc_err = rel(yff), rel(ytc)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    ly.test_apply(seed, v, w, ly.BF16_IR)
    ly.test_apply(seed, v, w, ly.TEST_FF)
    ly.test_apply(seed, v, w, ly.TEST_TC)
    ly.test_apply(seed, v, w, ly.FP64)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    pk, how = peaks()
    out = {}
    for name, d in prof.items():
        sec = d["total_ms"] / 1e3
        out[name] = dict(launches=d["launches"], avg_ms=d["total_ms"] / d["launches"],
                         tflops=d["flops"] / sec / 1e12 if d["flops"] else None,
                         gbs=d["bytes"] / sec / 1e9 if d["bytes"] else None)
    print(json.dumps(dict(probe="operators on 1000 systems, 800-state seed", kernels=out,
                          ff_max_rel_err_vs_fp64=ff_err, tc_max_rel_err_vs_fp64=tc_err,
                          bf16_peak_tflops=pk["bf16_tflops"],
                          peak_source=how)), flush=True)


def whole_job_rate(local_ms: float, units_per_rank: int, steps: int, dist=None, device=None):
    """Units per second over all ranks and the time it is taken over.

    Every rank processes units_per_rank units per step (independent replicas,
    weak scaling); the time is the slowest rank's (max over ranks).
    """
    total_ms = float(local_ms)
    world = 1
    if dist is not None:
        import torch

        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        world = dist.get_world_size()
    return world * units_per_rank * steps / (total_ms / 1000.0), total_ms


# -------------------------------------------------------------------- ours
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "serving":
        return run_serving(args, local) if rank == 0 else None
    if args.workload == "kernels":
        return run_kernel_probe(args, local) if rank == 0 else None

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    import paper_2312_08201_gb300 as ly
    from workloads import workload_precision

    ly.build()
    p, vs = workload_precision()
    if args.nv:
        vs = vs[: args.nv]
    nv, k = vs.shape
    ctx = ly.Context(local)
    seed = ly.Seed(ctx, p.A0, p.U, p.V, p.G, p.E)
    stats = seed.stats()
    dev = torch.device("cuda", local)
    v_dev = torch.tensor(vs, dtype=torch.float64, device=dev)

    precision = args.precision
    if precision == "best":
        precision = "bf16_ir" if _mixed_available(seed, v_dev) else "fp64"
    opts = dict(precision=ly.BF16_IR if precision == "bf16_ir" else ly.FP64, batch=args.batch)
    if args.pbar >= 0:
        opts["pbar"] = args.pbar
    if args.s >= 0:
        opts["s"] = args.s
    if precision == "bf16_ir":
        opts["residual"] = {"ff": ly.RESID_FF, "fp64": ly.RESID_FP64, "tc": ly.RESID_TC}[args.residual]

    # reference values of the FP64 GPU path (outside the timed region)
    f64 = seed.trace_EX(v_dev, precision=ly.FP64).cpu().numpy()

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        seed.trace_EX(v_dev, **opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream(dev)

    def timed_steps():
        # the per-system status records (return_info) are Python objects built
        # after the call returns; the timed steps do without them, as the
        # end-to-end measurement below does
        evs, outs = [], []
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()  # evict L2 (256 MiB write) between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f = seed.trace_EX(v_dev, **opts)
            e1.record(stream)
            evs.append((e0, e1))
            outs.append(f)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], outs

    # timed region: kernel accounting off (its events would add host work)
    step_ms, outs = timed_steps()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    # the same steps again with per-kernel CUDA-event accounting, for the
    # kernel shares and the roofline of the dominant kernel
    ly.prof_enable(True)
    prof_step_ms, _ = timed_steps()
    prof, launches = ly.prof_read()
    ly.prof_enable(False)
    value, total_ms = whole_job_rate(sum(step_ms), nv, args.steps, dist, dev)

    f_last = outs[-1].cpu().numpy()
    acc = np.abs(f_last - f64) / np.abs(f64)
    # iteration counts of one more sweep (untimed) of the same state
    _, info = seed.trace_EX(v_dev, return_info=True, **opts)
    iters = [i["iters"] for i in info]
    rsteps = [i["refine_steps"] for i in info]

    # end to end through the public API with host buffers (pinned inputs)
    v_pin = torch.from_numpy(vs.copy()).pin_memory()
    v_host = v_pin.numpy()
    seed.trace_EX(v_host, **opts)
    torch.cuda.synchronize()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()  # the same L2 state as the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fh = seed.trace_EX(v_host, **opts)
        e2e_s += time.perf_counter() - t0
    e2e = dict(value=nv * args.steps / e2e_s, unit="evals/s", h2d_bytes_per_step=int(nv * k * 8),
               d2h_bytes_per_step=int(nv * 8))

    # roofline of the dominant kernel (largest device time in the timed region)
    pk, how = peaks()
    dom_name = max(prof, key=lambda kname: prof[kname]["total_ms"]) if prof else None
    roof = None
    if dom_name:
        d = prof[dom_name]
        sec = d["total_ms"] / 1000.0
        if dom_name == "capmv64":
            sm_clock = float(pk.get("sm_max_mhz", 2070.0))
            peak = FP64_PEAK_FLOPS_PER_CLK_SM * SMS * sm_clock * 1e6 / 1e12
            ach = d["flops"] / sec / 1e12
            roof = dict(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=None,
                        kernel=dom_name, peak_source="FP64 FMA pipe: 152 SMs x 4 flop/clk x max SM clock",
                        launches=d["launches"], avg_launch_ms=d["total_ms"] / d["launches"])
        elif dom_name == "capmv_ff":
            sm_clock = float(pk.get("sm_max_mhz", 2070.0))
            peak = FP32_LANES_PER_SM * SMS * sm_clock * 1e6 / 1e12
            ach = d["flops"] / sec / 1e12
            roof = dict(bound="alu", achieved=ach, peak=peak, unit="Tinst/s", frac=ach / peak, traffic=None,
                        kernel=dom_name,
                        peak_source="FP32 pipe: 152 SMs x 128 lane-instructions/clk x max SM clock "
                                    "(achieved: 49.5 FP32 instructions per float-float complex MAC)",
                        launches=d["launches"], avg_launch_ms=d["total_ms"] / d["launches"])
        elif dom_name in ("tc_gemm", "oz_gemm", "prec_gemm"):
            peak = float(pk["bf16_tflops_sustained"])
            ach = d["flops"] / sec / 1e12
            roof = dict(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=None,
                        kernel=dom_name, peak_source=f"bf16 sustained ({how})", launches=d["launches"],
                        avg_launch_ms=d["total_ms"] / d["launches"])
        else:
            peak = float(pk["hbm_gbs"])
            ach = d["bytes"] / sec / 1e9
            roof = dict(bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak, traffic=None,
                        kernel=dom_name, peak_source=f"hbm copy ({how})", launches=d["launches"],
                        avg_launch_ms=d["total_ms"] / d["launches"])
    if roof is not None:
        d = prof[dom_name]
        roof["algorithmic_bytes_per_launch"] = d["bytes"] / d["launches"]
        if dom_name in MEASURED_TRAFFIC_PER_LAUNCH and precision == "bf16_ir" and nv == 1000:
            roof["traffic"] = MEASURED_TRAFFIC_PER_LAUNCH[dom_name]
            roof["traffic_note"] = ("DRAM bytes per launch, mean over the kernel's launches in one sweep, "
                                    "from a one-kernel ncu capture (1 pass)")
    kernels = {kname: dict(launches=v["launches"], ms=round(v["total_ms"], 3),
                           share=round(v["total_ms"] / max(1e-9, sum(x["total_ms"] for x in prof.values())), 4))
               for kname, v in prof.items()}

    line = dict(
        metric=METRIC, value=value, unit="evals/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f64" if precision == "fp64" else
        "bf16x3-gemm/f32-krylov/" + {"ff": "ff-refine", "fp64": "f64-refine", "tc": "int-sliced-bf16-refine"}[args.residual],
        data="synthetic",
        config=dict(workload=WORKLOAD, n=int(p.n), k=int(k), nv=int(nv), precision=precision, batch=args.batch,
                    pbar=int(ly.default_opts(**opts).pbar),
                    residual=args.residual if precision == "bf16_ir" else "fp64",
                    l2="flushed between steps (256 MiB device write outside the timed events)",
                    parallelism="replicas" if world > 1 else "single-gpu", cond_Q=stats["cond_Q"]),
        accuracy=dict(max_rel_err_vs_fp64_path=float(acc.max()), median_rel_err=float(np.median(acc)),
                      iters_mean=float(np.mean(iters)), refine_steps_mean=float(np.mean(rsteps))),
        sweep_ms=dict(p50=float(np.percentile(step_ms, 50)), p99=float(np.percentile(step_ms, 99)),
                      note="device time of one 1000-vector sweep"),
        roofline=roof, kernels=kernels, e2e=e2e, gpu_launches=int(launches), clocks=clk,
        profiled_ms_per_step=float(np.mean(prof_step_ms)),
        profile_note="kernel times, launches and roofline come from a second run of the same K steps "
                     "with per-kernel CUDA events; value is timed without them")

    if rank == 0 and world == 1 and not args.no_extras:
        # the figures of the other workloads, after the timed region
        for key, fn in (("fp64_path", lambda: extra_fp64_path(seed, v_dev, f64, stream)),
                        ("grad", lambda: extra_grad(ctx, dev, stream)),
                        ("multi_agent", lambda: extra_multi_agent(ctx, dev, stream)),
                        ("ex3", lambda: extra_ex3(ctx, dev, stream))):
            try:
                line[key] = fn()
            except Exception as exc:  # report, never lose the headline line
                line[key] = dict(error=f"{type(exc).__name__}: {exc}"[:300])
        try:
            sv = serving_measure(ctx, ly.BF16_IR, requests=args.serving_requests, fracs=(0.95,), burst=64)
            r = sv["rates"]["0.95"]
            line["serving"] = sv
            line["latency_ms"] = dict(p50=r["p50_ms"], p99=r["p99_ms"],
                                      request="one 64-vector request of the serving workload, submit to result, "
                                              "Poisson arrivals at 0.95 of measured saturation")
        except Exception as exc:
            line["serving"] = dict(error=f"{type(exc).__name__}: {exc}"[:300])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, fcpu, secs = cpu_oracle(args.cpu_sample)
        err = max(abs(a - b) / abs(b) for a, b in zip(f_last[: len(fcpu)], fcpu))
        line["cpu_baseline"] = dict(value=rate, unit="evals/s", cores=cores, kind="oracle",
                                    sample=f"first {len(fcpu)} of the 1000 parameter pairs, {secs:.1f} s",
                                    max_rel_err_gpu_vs_oracle=err)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if args.profile_sweep:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        seed.trace_EX(v_dev, **opts)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if dist:
        dist.destroy_process_group()


def _mixed_available(seed, v_dev):
    import paper_2312_08201_gb300 as ly

    try:
        seed.trace_EX(v_dev[:2], precision=ly.BF16_IR)
        return True
    except ly.LyapError:
        return False


if __name__ == "__main__":
    main()
