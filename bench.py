#!/usr/bin/env python
"""Benchmark of the preconditioned Legendre-Galerkin solve on one GB300 (or N replicas).

One step = the whole hot path on one synthetic problem: setup from the
coefficient samples (Gauss tables, truncated series, band matrices, M, ILU(0)),
the load vector, and PCG (Algorithm 1) to relative residual 1e-12 -- the 2D
FP64 workload N=512 (261,121 unknowns), T=8, a=exp(g_a), b=exp(g_b) random
Legendre series (seeds 1, 2), f with random Legendre coefficients (seed 3).
`value` is solves/s over all ranks with inputs resident in HBM; `e2e` is the
same through the C ABI with host buffers (copies inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun every rank solves its own replica (independent problems shard
with no data-path collective: weak scaling); timing is the max over ranks.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & A*x GDOF/s at rel. residual 1e-10 (mixed vs FP64); p50/p99 latency"
RTOL = 1e-12
WORKLOAD = "2d-exp-series N=512 (261,121 unknowns) T=8 Q=514, FP64 PCG+ILU(0) to rel. residual 1e-12"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, bf16 = 6800.0, 1900.0
    src = "fallback"
    if os.path.exists(path):
        with open(path) as fh:
            P = json.load(fh)
        hbm = float(P.get("hbm_gbs", hbm))
        bf16 = float(P.get("bf16_tflops", bf16))
        src = "measured"
    return hbm, bf16, src


# FP64 FMA throughput of this machine's GB300 (152 SMs): 1.194 TFLOP/s measured with an
# 8-chain DFMA loop over 8 CTAs/SM (0.5 of a DFMA per SM per clock at ~1.99 GHz).
FP64_PEAK_TFLOPS = 1.194

# ncu dram__bytes_read.sum + dram__bytes_write.sum per k_sweep_line launch (mean of the forward
# and backward sweep), 2D N=512 T=8 FP64, and the SHA-256 prefix of the sweep sources the counters
# were taken on: the figure is reported only while the kernel source is unchanged.
SWEEP_TRAFFIC = dict(bytes=475.61e6, source_sha="e4c3592c836f4f7d")


def sweep_source_sha():
    """Hash of the sweep kernels' source: sweep.cu up to its dispatch functions (which choose
    among preconditioners, not how a sweep runs), and stencil.cuh."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2004_13961_gb300", "csrc")
    with open(os.path.join(csrc, "sweep.cu")) as fh:
        txt = fh.read()
    h.update(txt[:txt.index("// FP64 vectors: FP64 factors with FP64 accumulation")].encode())
    with open(os.path.join(csrc, "stencil.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.out.name)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    samples=len(sm), reasons=sorted(reasons))


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- oracle (CPU) leg

def oracle_solve(p, rtol=RTOL):
    """One complete solve by the CPU oracle, timed: setup (truncated series, band matrices,
    M assembly, ILU(0) of Algorithm 2), the load vector by quadrature, and PCG (Algorithm 1)
    to the relative residual rtol -- the same steps the GPU step times."""
    import oracle as O
    d, N, T, Q = p["d"], p["N"], p["T"], p["Q"]
    t0 = time.perf_counter()
    F = O.load_vector(d, N, Q, p["f"])
    st = O.setup(d, N, Q, T, p["a"], p["b"])
    t1 = time.perf_counter()
    out = O.pcg(d, N, Q, p["a"], p["b"], st["LU"], F, eps=rtol)
    t2 = time.perf_counter()
    return dict(t_setup=t1 - t0, t_pcg=t2 - t1, t_solve=t2 - t0, iters=out["iters"], x=out["x"],
                relres_true=out["relres_true"], status=out["status"])


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    """The oracle on the host cores: every step (warm-up and timed) is one complete oracle solve
    of the workload (setup, load vector, PCG to 1e-12), timed with the host clock."""
    from paper_2004_13961_gb300 import workloads as W
    if rank != 0:
        return
    import oracle as O
    O.build()
    p = W.exp_2d_n512()
    for _ in range(args.warmup):
        oracle_solve(p)
    times, last = [], None
    for _ in range(args.steps):
        last = oracle_solve(p)
        times.append(last["t_solve"])
    t = float(np.mean(times))
    value = 1.0 / t
    cb = dict(value=value, unit="solves/s", cores=cores(), kind="oracle",
              sample=(f"per step one complete oracle solve at N=512: setup {last['t_setup']:.1f} s (truncated "
                      f"series, M assembly, ILU(0)), PCG {last['t_pcg']:.1f} s ({last['iters']} iterations to "
                      f"1e-12); mean of {args.steps} timed solves after {args.warmup} warm-up solves"))
    line = dict(metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=t * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference", config=dict(workload=WORKLOAD),
                cpu_baseline=cb, e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- native (GPU) leg

def run_batched(lsg, W, torch, dev, world, count=256, precision=None, threads=8):
    """Config 4: 256 independent 2D problems, N uniform on {32, 48, ..., 256} (seed 21), T=8,
    PCG to 1e-10 through lsg_batch_solve (FP64: one CUDA graph, every problem's loop on the
    device; mixed: concurrent refined solves).  Timed: setup of every context (ILU(0)
    included, `threads` host threads with a stream each) plus the batched solve."""
    from concurrent.futures import ThreadPoolExecutor
    precision = lsg.FP64 if precision is None else precision
    probs = W.batch_problems(count)
    dofs = sum((p["N"] - 1) ** 2 for p in probs)
    dev_in = [(torch.tensor(p["a"], device=dev), torch.tensor(p["b"], device=dev), torch.tensor(p["f"], device=dev))
              for p in probs]
    streams = [torch.cuda.Stream(device=dev) for _ in range(threads)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    def setup(k):
        out = []
        st = streams[k]
        for idx in range(k, count, threads):
            p = probs[idx]
            a, b, f = dev_in[idx]
            c = lsg.Context(2, p["N"], p["T"], a, b, allow_breakdown=True, precision=precision, stream=st,
                            shared_gpu=True)
            if c.status == lsg.ERR_ILU_BREAKDOWN:  # ILU(0) of this M does not exist: counted, not solved
                c.close()
                out.append((idx, None, None))
                continue
            with torch.cuda.stream(st):
                F = c.load_vector(f, stream=st)
                u0 = torch.zeros_like(F)
            out.append((idx, c, (F, u0)))
        st.synchronize()
        return out

    with ThreadPoolExecutor(threads) as ex:
        parts = [r for part in ex.map(setup, range(threads)) for r in part]
    parts.sort(key=lambda r: r[0])
    breakdowns = sum(1 for r in parts if r[1] is None)
    ctxs = [r[1] for r in parts if r[1] is not None]
    Fs = [r[2][0] for r in parts if r[1] is not None]
    us = [r[2][1] for r in parts if r[1] is not None]
    t1 = time.perf_counter()
    st, infos = lsg.batch_solve(ctxs, Fs, us, rtol=1e-10)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for c in ctxs:
        c.close()
    ok = sum(1 for i in infos if i["status"] == 0)
    total = max_over_ranks(t2 - t0, world)
    return dict(problems=count, converged=ok, ilu_breakdown=breakdowns, dof_total=dofs, rtol=1e-10,
                precision={lsg.FP64: "fp64", lsg.MIXED_TF32: "mixed-tf32", lsg.MIXED_BF16: "mixed-bf16"}[precision],
                setup_s=t1 - t0, solve_s=t2 - t1, solves_s=world * ok / total,
                gdof_s=world * dofs / total / 1e9, iters_mean=float(np.mean([i["iters"] for i in infos])),
                note=("setup on %d host threads; " % threads)
                + ("one CUDA graph launch, every problem's PCG loop in a device-side WHILE node"
                   if precision == lsg.FP64 else "concurrent refined solves, 8 host threads / streams"))


def _serve_once(lsg, W, data, rate_hz, precision, budget, inflight, world):
    """Submit the requests of `data` with Poisson arrivals at rate_hz (times scaled from the
    unit-rate draws), drain, and summarise latencies per class."""
    srv = lsg.Server(budget, max_inflight=inflight)
    rejected = 0
    t0 = time.perf_counter()
    for i, (r, p) in enumerate(data):
        delay = r["arrival_unit"] / rate_hz - (time.perf_counter() - t0) if rate_hz else 0.0
        if delay > 0:
            time.sleep(delay)
        st = srv.submit(i, r["d"], r["N"], r["T"], p["a"], p["b"], p["f"], precision=precision, rtol=1e-10)
        if st == lsg.ERR_NOMEM:
            rejected += 1
    srv.drain()
    t1 = time.perf_counter()
    res = srv.poll(len(data) + 8)
    srv.close()
    st = [x["info"]["status"] for x in res]
    out = dict(requests=len(data), handled=len(res), completed=int(sum(1 for v in st if v == 0)),
               ilu_breakdown=int(sum(1 for v in st if v == lsg.ERR_ILU_BREAKDOWN)),
               rejected_over_budget=rejected, other_errors=int(sum(1 for v in st if v not in (0, lsg.ERR_ILU_BREAKDOWN))),
               wall_s=t1 - t0, arrival_rate_hz=rate_hz)
    out["solves_s"] = world * out["completed"] / max_over_ranks(t1 - t0, world)
    out["handled_s"] = out["handled"] / (t1 - t0)
    lat = np.array([x["latency_ms"] for x in res if x["info"]["status"] == 0])
    if len(lat):
        out.update(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)))
    by = {}
    for dd in (2, 3):
        l = np.array([x["latency_ms"] for x in res if x["info"]["status"] == 0 and data[x["id"]][0]["d"] == dd])
        c = dict(requests=sum(1 for r, _ in data if r["d"] == dd), completed=int(len(l)))
        if len(l):
            c.update(p50_ms=float(np.percentile(l, 50)), p99_ms=float(np.percentile(l, 99)))
        by[f"{dd}d"] = c
    out["by_class"] = by
    return out


def run_serving(lsg, W, world, precision, count=40, n2d=(64, 1024), n3d=(24, 40), budget_gb=64, inflight=4,
                fracs=(0.5, 0.8, 0.95), rates=None):
    """Config 5 (serving) as continuous batching: requests of the mix (70% 2D, N log-uniform in
    n2d; 30% 3D, N uniform in n3d; T in {4, 8}; a = exp(g) with sigma in [0.5, 2.3]; refined to
    1e-10) admitted by HBM footprint into `inflight` slots.  First the capacity mu: every
    request at t = 0, mu = requests handled per second; then Poisson arrivals at 0.5, 0.8 and
    0.95 mu.  Latency runs from submit to the solution in host memory."""
    reqs = W.serving_stream(count, seed=31, rate_hz=1.0, n2d=n2d, n3d=n3d)
    data = []
    for r in reqs:
        p = W.random_exp_problem(r["d"], r["N"], r["T"], r["seed"], r["seed"] + 1, r["seed"] + 2, sigma=r["sigma"])
        r = dict(r, arrival_unit=r["arrival_s"])
        data.append((r, p))
    budget = int(budget_gb) << 30
    sat = _serve_once(lsg, W, data, 0.0, precision, budget, inflight, world)
    mu = sat["handled_s"]
    runs = {"saturated": sat}
    for f in fracs:
        runs[f"{f:.2f}mu"] = _serve_once(lsg, W, data, f * mu, precision, budget, inflight, world)
    for name, rate in (rates or {}).items():
        runs[name] = _serve_once(lsg, W, data, rate, precision, budget, inflight, world)
    return dict(precision="mixed-tf32" if precision == lsg.MIXED_TF32 else "fp64", rtol=1e-10, capacity_mu=mu,
                hbm_budget_gb=budget_gb, slots=inflight,
                sample=(f"{count} requests of the config-5 mix per run (2D N in [{n2d[0]}, {n2d[1]}], 3D N in "
                        f"[{n3d[0]}, {n3d[1]}]); the same requests at every rate"), runs=runs)


def run_serving_large(lsg, W, world, precision, budget_gb=64):
    """The config-5 sizes at the top of its range, each served alone through the same server:
    2D N=1024 T=8, 3D N=128 and N=160 with T=4 (sigma 0.5, seeds of the 3D configuration), and
    3D N=160 T=8, whose FP32 factors (~135 GB) exceed the HBM budget and are rejected at submit
    (LSG_ERR_NOMEM)."""
    cases = [(2, 1024, 8), (3, 128, 4), (3, 160, 4), (3, 160, 8)]
    out = []
    for d, N, T in cases:
        fp = lsg.footprint_bytes(d, N, T, N + 2, precision)
        row = dict(d=d, N=N, T=T, footprint_gb=fp / 2 ** 30)
        if fp > (budget_gb << 30):
            srv = lsg.Server(budget_gb << 30, max_inflight=1)
            one = np.ones(1)
            nq = (N + 2) ** d
            z = np.ones(nq)
            row["submit_status"] = srv.submit(0, d, N, T, z, z, z, precision=precision)
            srv.close()
            out.append(row)
            continue
        # 3D: the seeds of the 3D configuration (11-13), whose degree-4 preconditioner factorises
        seeds = (11, 12, 13) if d == 3 else (777 + N, 778 + N, 779 + N)
        p = W.random_exp_problem(d, N, T, *seeds, sigma=0.5)
        data = [(dict(d=d, N=N, T=T, arrival_unit=0.0), p)]
        r = _serve_once(lsg, W, data, 0.0, precision, budget_gb << 30, 1, world)
        row.update(status="ok" if r["completed"] else ("ilu_breakdown" if r["ilu_breakdown"] else "error"),
                   latency_ms=r.get("p50_ms"), wall_s=r["wall_s"])
        out.append(row)
    return out


def run_c3(lsg, W, torch, dev, world):
    """Config 3 (3D N=128): FP64 PCG to 1e-12 against the mixed form (TF32 and BF16 tensor-core
    products, FP32 ILU(0), FP64 refinement to 1e-10).  With the configuration's T = 6 the ILU(0)
    of M does not exist (non-positive pivots); the comparison runs on its stand-in with the same
    seeds (11-13) and series and truncation of degree 4, where it exists.  Each result states its
    true relative residual from the library's FP64 K x (which the tests pin to the oracle's at
    1e-11; the full-size test also checks these solves with the oracle's own K x)."""
    out = {}
    pc = W.exp_3d()
    c = lsg.Context(3, pc["N"], pc["T"], torch.tensor(pc["a"], device=dev), torch.tensor(pc["b"], device=dev),
                    precision=lsg.MIXED_TF32, allow_breakdown=True)
    out["t6_ilu_status"] = c.status
    c.close()
    p = W.random_exp_problem(3, 128, 4, 11, 12, 13)
    a, b, f = (torch.tensor(p[k], device=dev) for k in ("a", "b", "f"))
    sols = {}
    for name, prec, rtol in (("fp64", lsg.FP64, 1e-12), ("mixed_tf32", lsg.MIXED_TF32, 1e-10),
                             ("mixed_bf16", lsg.MIXED_BF16, 1e-10)):
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        ctx = lsg.Context(3, 128, 4, a, b, precision=prec, profile=True)
        F = ctx.load_vector(f)
        u, info = ctx.pcg_solve(F, rtol=rtol, check=False)
        s1.record()
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1)
        sols[name] = u.cpu().numpy()
        out[name] = dict(solves_s=1e3 / ms, ms_per_solve=ms, status=info["status"], iters=info["iters"],
                         refinements=info["outer_iters"], relres_true_fp64=info["relres_true"],
                         setup_ms=dict(assemble=ctx.query(lsg.Q_ASSEMBLE_US) / 1e3, ilu=ctx.query(lsg.Q_ILU_US) / 1e3),
                         sweeps_ms=(ctx.query(lsg.Q_SWEEP_L_US) + ctx.query(lsg.Q_SWEEP_U_US)) / 1e3,
                         sweep_launches=ctx.query(lsg.Q_SWEEP_L_CALLS) + ctx.query(lsg.Q_SWEEP_U_CALLS),
                         kx_ms=(ctx.query(lsg.Q_KX_US) + ctx.query(lsg.Q_KX_LO_US)) / 1e3,
                         device_gb=ctx.query(lsg.Q_DEVICE_BYTES) / 2 ** 30)
        ctx.close()
    x64 = sols["fp64"]
    for name in ("mixed_tf32", "mixed_bf16"):
        out[name]["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(sols[name] - x64) / np.linalg.norm(x64))
    out["workload"] = ("3D N=128 (2,048,383 unknowns), Q=130, seeds 11-13; T=6 (the configuration): ILU(0) "
                       "breaks down; compared at T=4 with degree-4 series")
    return out


def run_native(args, world, rank, local):
    import torch
    from paper_2004_13961_gb300 import lsg
    from paper_2004_13961_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lsg.load()
    p = W.exp_2d_n512()
    d, N, T, Q = p["d"], p["N"], p["T"], p["Q"]
    a = torch.tensor(p["a"], device=dev)
    b = torch.tensor(p["b"], device=dev)
    f = torch.tensor(p["f"], device=dev)
    n = (N - 1) ** d
    F = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2 (129 MB)

    last = {}
    prof = dict(sweep_us=0.0, sweep_calls=0, sweep_l_calls=0, kx_us=0.0, kx_calls=0, ilu_us=0.0, asm_us=0.0)

    def step(timed=False):
        # the context records CUDA events on its stream around every sweep and K x kernel
        ctx = lsg.Context(d, N, T, a, b, Q=Q, profile=True)
        ctx.load_vector(f, F)
        u.zero_()
        _, info = ctx.pcg_solve(F, u, rtol=RTOL)
        last["info"] = info
        last["ilu_ms"] = ctx.query(lsg.Q_ILU_US) / 1e3
        last["asm_ms"] = ctx.query(lsg.Q_ASSEMBLE_US) / 1e3
        if timed:
            prof["sweep_us"] += ctx.query(lsg.Q_SWEEP_L_US) + ctx.query(lsg.Q_SWEEP_U_US)
            prof["sweep_calls"] += ctx.query(lsg.Q_SWEEP_L_CALLS) + ctx.query(lsg.Q_SWEEP_U_CALLS)
            prof["sweep_l_calls"] += ctx.query(lsg.Q_SWEEP_L_CALLS)
            prof["kx_us"] += ctx.query(lsg.Q_KX_US)
            prof["kx_calls"] += ctx.query(lsg.Q_KX_CALLS)
            prof["ilu_us"] += ctx.query(lsg.Q_ILU_US)
            prof["asm_us"] += ctx.query(lsg.Q_ASSEMBLE_US)
        ctx.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    l0 = lsg.kernel_launches()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict L2 between timed steps (outside the events)
        ev[k][0].record()
        step(timed=True)
        ev[k][1].record()
    torch.cuda.synchronize()
    launches = lsg.kernel_launches() - l0
    clocks = sampler.stop()
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in ev]
    t_total = max_over_ranks(sum(step_ms) / 1e3, world)
    value = world * args.steps / t_total
    info = last["info"]

    # ---- stage breakdown (separate from the timed steps) ----
    ctx = lsg.Context(d, N, T, a, b, Q=Q)
    ctx.load_vector(f, F)
    x = torch.randn(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)

    def evtime(fn, reps):
        fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    t_kx = evtime(lambda: ctx.apply_A(x, y), 20)
    t_minv = evtime(lambda: ctx.apply_Minv(F, z), 3)
    nnz = ctx.query(lsg.Q_NNZ)
    ctx.close()
    hbm, bf16, psrc = peaks()
    n1 = N - 1
    # algorithmic work (per launch): a sweep reads its triangle of M's structural
    # nonzeros (forward: strictly lower, backward: diagonal and upper) plus the
    # right-hand side and writes its result, all FP64; a K x does the parity-folded
    # 2D contractions (8 n1^2 Q + 12 Q^2 n1) / 2 flops
    sweep_bytes_total = 8.0 * (prof["sweep_l_calls"] * ((nnz - n) / 2 + 2 * n)
                               + (prof["sweep_calls"] - prof["sweep_l_calls"]) * ((nnz + n) / 2 + 2 * n))
    kx_flops = (8.0 * n1 * n1 * Q + 12.0 * Q * Q * n1) / 2.0
    stage_ms = dict(sweeps=prof["sweep_us"] / 1e3, kx=prof["kx_us"] / 1e3, ilu=prof["ilu_us"] / 1e3,
                    assemble=prof["asm_us"] / 1e3)
    dominant = max(stage_ms, key=stage_ms.get)
    if dominant == "sweeps":
        dur_s = prof["sweep_us"] / 1e6 / max(1, prof["sweep_calls"])
        # DRAM bytes per sweep launch measured by ncu on this workload, valid only for the
        # sweep source it was taken on
        traffic = (SWEEP_TRAFFIC["bytes"] if (d, N, T) == (2, 512, 8)
                   and SWEEP_TRAFFIC["source_sha"] == sweep_source_sha() else None)
        roof = dict(kernel="k_sweep_line (one triangular sweep, Algorithm 3 or 4; timed with its output fill)",
                    bound="hbm",
                    achieved=sweep_bytes_total / max(1, prof["sweep_calls"]) / dur_s / 1e9, peak=hbm, unit="GB/s",
                    launches=prof["sweep_calls"], avg_launch_ms=dur_s * 1e3, traffic=traffic,
                    check_minv_half_ms=t_minv / 2,
                    algorithmic_bytes_per_launch=sweep_bytes_total / max(1, prof["sweep_calls"]))
    elif dominant == "kx":
        dur_s = prof["kx_us"] / 1e6 / max(1, prof["kx_calls"])
        roof = dict(kernel="K x (k_xf_fwd + k_xf_bwd, FP64)", bound="alu", achieved=kx_flops / dur_s / 1e12,
                    peak=FP64_PEAK_TFLOPS, unit="TFLOP/s", launches=prof["kx_calls"], avg_launch_ms=dur_s * 1e3,
                    traffic=None)
    else:
        roof = dict(kernel="k_ilu0 (Algorithm 2)", bound="alu", achieved=None, peak=FP64_PEAK_TFLOPS,
                    unit="TFLOP/s", traffic=None)
    if roof["achieved"] is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_source"] = ("of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if psrc == "measured"
                           else "of fallback") if roof["bound"] == "hbm" else "of measured FP64 FMA loop"
    roof["timing"] = ("CUDA events on the launching stream around every launch of the timed steps that did "
                      "work (launches queued after the stop test return at once and are not counted)")
    iters = info["iters"]
    per_solve = {k + "_ms": v / args.steps for k, v in stage_ms.items()}

    # ---- mixed precision: inner FP32 PCG (FP32 ILU factors, FP32 transforms) in FP64 refinement ----
    mixed, mixed_u = {}, {}
    if not args.no_mixed:
        u64 = u.clone()
        for name, prec in (("tf32", lsg.MIXED_TF32), ("bf16", lsg.MIXED_BF16)):
            um = torch.empty_like(u)
            res = {}

            def mstep():
                c3 = lsg.Context(d, N, T, a, b, Q=Q, precision=prec, profile=True)
                c3.load_vector(f, F)
                um.zero_()
                _, inf = c3.pcg_solve(F, um, rtol=1e-10)
                res["info"] = inf
                res["stages"] = dict(ilu_ms=c3.query(lsg.Q_ILU_US) / 1e3,
                                     sweeps_ms=(c3.query(lsg.Q_SWEEP_L_US) + c3.query(lsg.Q_SWEEP_U_US)) / 1e3,
                                     kx_tensor_core_ms=c3.query(lsg.Q_KX_LO_US) / 1e3,
                                     kx_tensor_core_calls=c3.query(lsg.Q_KX_LO_CALLS))
                c3.close()

            for _ in range(2):
                mstep()
            torch.cuda.synchronize()
            ms = []
            for k in range(max(1, min(args.steps, 3))):
                flush.fill_(float(k))
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                mstep()
                s1.record()
                torch.cuda.synchronize()
                ms.append(s0.elapsed_time(s1))
            inf = res["info"]
            mixed_u[name] = um.cpu().numpy()
            err = float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64))
            mixed[name] = dict(solves_s=world * 1e3 / max_over_ranks(float(np.mean(ms)), world),
                               ms_per_solve=float(np.mean(ms)), rtol=1e-10, relres_true=inf["relres_true"],
                               inner_iters=inf["iters"], refinements=inf["outer_iters"],
                               rel_err_vs_fp64_gpu=err, stages_last_solve=res["stages"],
                               transforms=f"tcgen05 tensor cores, {name.upper()} operands split hi+lo (3 MMAs), FP32 accumulation")

    # ---- e2e: host buffers through the C ABI, copies inside the timed region ----
    ha, hb, hf = p["a"].copy(), p["b"].copy(), p["f"].copy()
    hF = np.empty(n)
    hu = np.empty(n)
    e2e_t = []
    for k in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = lsg.Context(d, N, T, ha, hb, Q=Q)
        c2.load_vector(hf, hF)
        hu[:] = 0.0
        c2.pcg_solve(hF, hu, rtol=RTOL)
        c2.close()
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = world / max_over_ranks(float(np.mean(e2e_t)), world)
    nq = Q ** d
    e2e = dict(value=e2e_val, unit="solves/s", h2d_bytes_per_step=3 * nq * 8 + 2 * n * 8,
               d2h_bytes_per_step=2 * n * 8)

    batched = None if args.no_batch else dict(
        fp64=run_batched(lsg, W, torch, dev, world),
        mixed_tf32=run_batched(lsg, W, torch, dev, world, precision=lsg.MIXED_TF32))
    serving = None
    if not args.no_serving:
        mixed_srv = run_serving(lsg, W, world, lsg.MIXED_TF32)
        # plain FP64 on the same requests: its own capacity, and the mixed form's 0.5 mu load
        fp64_srv = run_serving(lsg, W, world, lsg.FP64, fracs=(),
                               rates={"mixed_0.50mu": 0.5 * mixed_srv["capacity_mu"]})
        serving = dict(mixed_tf32=mixed_srv, fp64=fp64_srv,
                       large_mixed_tf32=run_serving_large(lsg, W, world, lsg.MIXED_TF32))
    c3 = None if args.no_c3 else run_c3(lsg, W, torch, dev, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        o = oracle_solve(p)
        cpu = dict(value=1.0 / o["t_solve"], unit="solves/s", cores=cores(), kind="oracle",
                   sample=(f"one complete oracle solve at N=512: setup {o['t_setup']:.1f} s (load vector, truncated "
                           f"series, M assembly, ILU(0)), PCG {o['t_pcg']:.1f} s ({o['iters']} iterations to 1e-12)"),
                   iters=o["iters"])
        # the GPU results against the FP64 oracle's solution of the same problem
        xo = o["x"]
        cpu["rel_err_fp64_gpu_vs_oracle"] = float(np.linalg.norm(u.cpu().numpy() - xo) / np.linalg.norm(xo))
        for name, um in mixed_u.items():
            mixed[name]["rel_err_vs_fp64_oracle"] = float(np.linalg.norm(um - xo) / np.linalg.norm(xo))

    if rank == 0:
        line = dict(
            metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=t_total * 1e3 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f64", data="synthetic",
            config=dict(workload=WORKLOAD, l2="256 MB buffer written between timed steps (factors 0.94 GB > L2)",
                        parallelism=f"replicas x{world}"),
            kx_gdof_s=n / (t_kx * 1e-3) / 1e9, kx_ms=t_kx, minv_ms=t_minv, pcg_iters=iters,
            relres_true=info["relres_true"], breakdown_ms_per_solve=per_solve, mixed=mixed or None,
            batched=batched, serving=serving, config3=c3,
            roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches, clocks=clocks)
        print(json.dumps(line), flush=True)


def run_profile_case(args):
    """One setup + solve of the 2D N=256, T=8 exp-series problem (seeds 1, 2, 3; factors
    ~0.23 GB, above L2): a small case for ncu captures of the sweep, ILU(0) and tensor-core kernels."""
    import torch
    from paper_2004_13961_gb300 import lsg
    from paper_2004_13961_gb300 import workloads as W
    lsg.load()
    dev = torch.device("cuda", 0)
    if args.profile_case == "n512-tf32-kx":
        # three tensor-core products K x at the bench workload's size (2D N=512 T=8, TF32)
        p = W.exp_2d_n512()
        a, b = torch.tensor(p["a"], device=dev), torch.tensor(p["b"], device=dev)
        ctx = lsg.Context(2, 512, 8, a, b, precision=lsg.MIXED_TF32)
        g = torch.Generator(device=dev).manual_seed(4)
        x = torch.randn(ctx.n, dtype=torch.float32, device=dev, generator=g)
        y = torch.empty_like(x)
        for _ in range(3):
            ctx.apply_A_lowp(x, y)
        torch.cuda.synchronize()
        print(json.dumps(dict(profile_case=args.profile_case, sum_abs=float(y.abs().sum()))), flush=True)
        ctx.close()
        return
    prec = {"n256-fp64": lsg.FP64, "n256-tf32": lsg.MIXED_TF32, "n256-bf16": lsg.MIXED_BF16}[args.profile_case]
    p = W.random_exp_problem(2, 256, 8, 1, 2, 3)
    a, b, f = (torch.tensor(p[k], device=dev) for k in ("a", "b", "f"))
    # profiled context: the host-driven PCG loop (kernels inside a graph's device-side loop
    # cannot be captured one by one)
    ctx = lsg.Context(2, 256, 8, a, b, precision=prec, profile=True)
    F = ctx.load_vector(f)
    u, info = ctx.pcg_solve(F, rtol=1e-12 if prec == lsg.FP64 else 1e-10)
    torch.cuda.synchronize()
    print(json.dumps(dict(profile_case=args.profile_case, info=info)), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the 3D N=128 FP64-vs-mixed line")
    ap.add_argument("--profile-case", choices=["n256-fp64", "n256-tf32", "n256-bf16", "n512-tf32-kx"], default=None,
                    help="run one 2D N=256 T=8 setup + solve (or three 2D N=512 tensor-core products) and exit: "
                         "the small cases of the ncu captures")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
