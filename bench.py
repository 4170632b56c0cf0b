"""Benchmark of the UBQP hot path on GB300: one JSON line on stdout (rank 0).

A step is one pass of the whole hot path over one batch of synthetic starts on
a device-resident instance: start generation, exact xQx evaluation of every
start, the T(lambda) screen, steepest ascent of the passing starts and the
best-of -- the loop body of Fig. 2 applied to a batch.  The default workload is
the Table 1 shape at its largest size: n = 7000, dense Q (density 1.0, integer
coefficients uniform in [-100, 100], seed 7000), 1000 uniformly random starts
per step (a new batch every step), lambda = 0.5.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own batches of the
same instance (weak scaling, no data-path collective); the time is the max over
ranks.  --impl reference times the CPU oracle (the reference arm of this
project) on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "xQx evals/s and 1-flip moves/s at n=7000; served solves/s with p50/p99 latency"
UNIT = "starts/s"  # starts taken through the whole round per second
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=7000)
    ap.add_argument("--density", type=float, default=1.0)
    ap.add_argument("--starts", type=int, default=1000)
    ap.add_argument("--lam", type=float, default=0.5)
    ap.add_argument("--eval-path", choices=["auto", "tc", "plain"], default="auto")
    ap.add_argument("--cpu-sample", type=int, default=160,
                    help="starts in the oracle's timed sample")
    ap.add_argument("--workload", choices=["table1", "batch64", "serve", "configs"],
                    default="table1",
                    help="table1: the default line; batch64: 64 uneven instances, batched "
                         "vs one at a time; serve: the request-serving loop; configs: "
                         "per-configuration measurements")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="seconds of Poisson arrivals (default 60 for --workload serve, 10 "
                         "inside the default line)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload_name(a):
    return f"table1-dense-n{a.n}" if a.density == 1.0 else f"n{a.n}-d{a.density}"


def config_of(a, world):
    return {"workload": workload_name(a), "n": a.n, "density": a.density,
            "coeffs": "int8 uniform [-100,100]", "instance_seed": a.n,
            "starts_per_step": a.starts, "start_mode": "RANDOM (new seed per step)",
            "lambda": a.lam, "max_flips": 0, "eval_path": a.eval_path,
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or self.path is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def profiled_traffic(summary: str, key: str):
    """DRAM bytes per launch recorded in a committed ncu summary, or None when
    the kernel's source changed since the capture (sha256 prefix recorded)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    val, src, digest = None, None, None
    for line in text.splitlines():
        if line.startswith(key + ":"):
            val = int(line.split(":")[1])
        if line.startswith("source:"):
            parts = line.split()
            src, digest = parts[1], parts[-1]
    if val is None or src is None:
        return None
    try:
        now = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return val if now == digest else None


# --------------------------------------------------------------------- oracle arm

def cpu_sample(a, Q, S_cpu, seed):
    """Whole path on the CPU oracle for S_cpu starts; returns (seconds, flips)."""
    import oracle as orc
    t0 = time.perf_counter()
    X = orc.diversify(None, a.n, orc.RANDOM, seed, 0, S_cpu)
    f = orc.eval(Q, X)
    sc = orc.screen(f, a.lam)
    _, f2, flips = orc.ascent(Q, X, f, sc["idx"])
    orc.best(f2)
    return time.perf_counter() - t0, int(flips.sum())


_ORACLE_Q = {}


def _oracle_worker_init(n, density, seed, ready=None):
    from paper_1706_00037_gb300 import synth
    _ORACLE_Q[n] = synth.make_instance(n, density, seed)
    if ready is not None:
        ready.wait()  # every worker holds the instance before any timing starts


def _oracle_ascent_chunk(args):
    """Climb a chunk of passing starts with the oracle in a pool worker."""
    import oracle as orc
    n, Xh, fh = args
    return orc.ascent(_ORACLE_Q[n], Xh, fh, np.arange(Xh.shape[0], dtype=np.int32))


class OraclePool:
    """One spawned process per host core, each holding its own copy of the
    seeded instance (built from its generator, not sent); ready when made."""

    def __init__(self, n, density, seed):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.n = n
        self.procs = os.cpu_count() or 1
        ready = ctx.Barrier(self.procs + 1)
        self.pool = ctx.Pool(self.procs, initializer=_oracle_worker_init,
                             initargs=(n, density, seed, ready))
        ready.wait()

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_sample_all_cores(op, a, S_cpu, seed):
    """The whole path on the oracle for S_cpu starts, spread over op's
    processes: the evaluation in equal chunks, the screen over the whole batch
    and the best-of here, the passing starts' ascents in small chunks taken as
    processes free up.  Returns (seconds, flips)."""
    import oracle as orc
    t0 = time.perf_counter()
    X = orc.diversify(None, a.n, orc.RANDOM, seed, 0, S_cpu)
    parts = [p for p in np.array_split(np.arange(S_cpu), op.procs) if len(p)]
    f = np.concatenate([r[0] for r in op.pool.map(_oracle_eval_chunk,
                                                   [(a.n, X[p]) for p in parts])])
    sc = orc.screen(f, a.lam)
    idx = np.asarray(sc["idx"], dtype=np.int64)
    chunks = [c for c in np.array_split(idx, 4 * op.procs) if len(c)]
    outs = op.pool.map(_oracle_ascent_chunk, [(a.n, X[c], f[c]) for c in chunks], chunksize=1)
    f2, flips = f.copy(), 0
    for c, (_, fc, flc) in zip(chunks, outs):
        f2[c] = fc
        flips += int(flc.sum())
    orc.best(f2)
    return time.perf_counter() - t0, flips


def _oracle_eval_chunk(args):
    """Evaluate a chunk of starts with the oracle in a pool worker; returns
    (values, seconds)."""
    import oracle as orc
    n, Xh = args
    t0 = time.perf_counter()
    f = orc.eval(_ORACLE_Q[n], Xh)
    return f, time.perf_counter() - t0


def oracle_eval_all_cores(n, density, seed, Xh):
    """The oracle's evaluation of the rows of Xh split over every host core
    (one spawned process per core, each holding its own copy of the seeded
    instance); returns (values, wall seconds of the evaluation, processes)."""
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    parts = np.array_split(Xh, procs)
    with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(n, density, seed)) as pool:
        pool.map(_oracle_eval_chunk, [(n, p[:1]) for p in parts])  # every worker ready
        t0 = time.perf_counter()
        out = pool.map(_oracle_eval_chunk, [(n, p) for p in parts])
        dt = time.perf_counter() - t0
    return np.concatenate([o[0] for o in out]), dt, procs


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    op = OraclePool(a.n, a.density, a.n)
    # per step each core takes the sample the single-thread arm took
    S_cpu = max(4, min(a.starts, a.cpu_sample // 8)) * op.procs
    try:
        for w in range(a.warmup):
            cpu_sample_all_cores(op, a, S_cpu, 10_000 + w)
        total = 0.0
        for k in range(a.steps):
            dt, _ = cpu_sample_all_cores(op, a, S_cpu, 20_000 + k)
            total += dt
    finally:
        op.close()
    value = S_cpu * a.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": dict(config_of(a, 1), starts_per_step=S_cpu),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.procs,
                             "kind": "oracle",
                             "sample": f"{S_cpu} random starts per step through the whole "
                                       f"path, spread over {op.procs} processes (one "
                                       f"per host core)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU arm

def batch_instances(count=64, seed=4):
    """64 instances: n ~ U[200, 2500], density in {0.1, 0.5, 1.0} (synth.batch_specs)."""
    from paper_1706_00037_gb300 import synth
    return [(n, d, synth.make_instance(n, d, s)) for n, d, s in synth.batch_specs(count, seed)]


def run_batch64(a):
    """Solves/s for 64 uneven instances: the batch plan (autotuned, CUDA graph)
    against solving the same instances one at a time through ubqp_solve."""
    import torch
    from paper_1706_00037_gb300 import ubqp
    torch.cuda.set_device(0)
    data = batch_instances()
    insts = [ubqp.Instance(torch.from_numpy(Q).cuda()) for _, _, Q in data]
    S, lam = 1024, 0.5
    params = ubqp.make_params(S, lam, seed=0)
    # one at a time, workspace reused
    need = max(ubqp.solve_workspace_size(i, params) for i in insts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    bx = [torch.empty(i.words, dtype=torch.int64, device="cuda") for i in insts]
    bf = [torch.empty(2, dtype=torch.int64, device="cuda") for _ in insts]

    def loop(seed):
        for k, inst in enumerate(insts):
            params.seed = seed
            ubqp.solve(inst, params, ws=ws, best_x=bx[k], best_f=bf[k], want_stats=False)

    for w in range(a.warmup):
        loop(10 + w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(a.steps):
        loop(100 + k)
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    ref = [(bf[k].clone(), bx[k].clone()) for k in range(len(insts))]
    # batched: tune, capture, replay
    b = ubqp.Batch(insts, ubqp.make_params(S, lam, seed=0))
    b.tune()
    b.capture()
    for w in range(a.warmup):
        b.run(10 + w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for k in range(a.steps):
        b.run(100 + k)
    e1.record()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    same = all(torch.equal(b.result(k)[1], ref[k][0]) and torch.equal(b.result(k)[0], ref[k][1])
               for k in range(len(insts)))
    value = len(insts) * a.steps / t_batch
    line = {"metric": "solves/s, 64 instances n~U[200,2500]", "value": value, "unit": "solves/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_batch / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batch64", "instances": len(insts),
                       "n": [n for n, _, _ in data], "starts_per_instance": S, "lambda": lam,
                       "batch_config": b.config()},
            "per_instance_loop_solves_per_s": len(insts) * a.steps / t_loop,
            "speedup_batched_vs_loop": t_loop / t_batch,
            "device_ms_per_batch": e0.elapsed_time(e1) / a.steps,
            "results_identical_to_loop": bool(same)}
    print(json.dumps(line), flush=True)


def serve_measure(duration_s: float, rate: float = 200.0, workers: int = 4, seed: int = 5,
                  seq_requests: int = 100, max_batch: int = 16):
    """Poisson arrivals at `rate` req/s for `duration_s` into the request loop,
    each request its own instance (synth.serve_requests: n log-uniform on
    [500, 7000], density in {0.1, 1.0}, a principal submatrix of a seeded
    n = 8192 master passed in place); returns served solves/s, latency
    percentiles, the saturated rate and the one-at-a-time rate."""
    import threading
    import torch
    from paper_1706_00037_gb300 import synth, ubqp
    masters_np = {d: synth.serve_master(d) for d in (0.1, 1.0)}
    masters = {d: torch.from_numpy(M).pin_memory() for d, M in masters_np.items()}
    S, lam = 1024, 0.5
    params = ubqp.make_params(S, lam, seed=0)
    r = np.random.default_rng(seed)
    gaps = r.exponential(1.0 / rate, int(rate * duration_s * 1.2) + 16)
    t_arr = np.cumsum(gaps)
    t_arr = t_arr[t_arr < duration_s]
    reqs = synth.serve_requests(len(t_arr) + 1200, seed)
    srv = ubqp.Server(workers, synth.SERVE_MASTER_N, params, max_batch=max_batch)
    for k in range(4 * workers):  # warm-up (module loading, pool growth)
        n, d, o = reqs[-1 - k]
        srv.wait(srv.submit(masters[d], 10**6 + k, n=n, offset=o))
    tickets = [None] * len(t_arr)
    t0 = time.perf_counter()

    def submitter():
        for k, ta in enumerate(t_arr):
            dly = t0 + ta - time.perf_counter()
            if dly > 0:
                time.sleep(dly)
            n, d, o = reqs[k]
            tickets[k] = srv.submit(masters[d], k, n=n, offset=o)

    st0 = srv.stats()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res = [srv.wait(t) for t in tickets]
    t_end = time.perf_counter()
    st1 = srv.stats()
    # capacity: the next requests of the mix submitted at once (a saturating burst)
    burst = 1200
    tb = time.perf_counter()
    bt = [srv.submit(masters[d], 2 * 10**6 + k, n=n, offset=o)
          for k, (n, d, o) in enumerate(reqs[len(t_arr):len(t_arr) + burst])]
    for t in bt:
        srv.wait(t)
    t_burst = time.perf_counter() - tb
    st2 = srv.stats()
    srv.close()
    lat = np.array([x[2] for x in res]) * 1e3
    # the first requests one at a time through the public API (upload,
    # prepare, ubqp_solve, result back), each from a contiguous pinned copy
    m = min(seq_requests, len(res))
    copies = [torch.from_numpy(np.ascontiguousarray(masters_np[d][o:o + n, o:o + n])).pin_memory()
              for n, d, o in reqs[:m]]
    same = True
    ts = time.perf_counter()
    for k in range(m):
        inst = ubqp.Instance(copies[k].to("cuda", non_blocking=True))
        params.seed = k
        bx, bf, _ = ubqp.solve(inst, params, want_stats=False)
        bfh = bf.cpu().tolist()
        same = same and bfh == res[k][0] and np.array_equal(
            bx.cpu().numpy().view(np.uint64), res[k][1])
        inst.close()
    t_seq = time.perf_counter() - ts
    ns = [n for n, _, _ in reqs[:len(t_arr)]]
    return {"served_solves_per_s": len(res) / (t_end - t0), "requests": len(res),
            "offered_req_per_s": rate, "duration_s": duration_s, "lanes": workers,
            "max_batch": max_batch,
            "mean_batch_served": (st1["requests"] - st0["requests"]) /
                                 max(st1["batches"] - st0["batches"], 1),
            "mean_batch_saturated": (st2["requests"] - st1["requests"]) /
                                    max(st2["batches"] - st1["batches"], 1),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()),
            "saturated_solves_per_s": burst / t_burst, "saturating_burst": burst,
            "sequential_solves_per_s": m / t_seq, "sequential_requests": m,
            "results_identical_to_alone": bool(same),
            "requests_mix": {"instances": "one per request: principal submatrix of a seeded "
                                          "n=8192 master at a random offset",
                             "n_mean": float(np.mean(ns)), "n_min": int(min(ns)),
                             "n_max": int(max(ns)), "starts": S, "lambda": lam}}


def run_serve(a):
    import torch
    torch.cuda.set_device(0)
    m = serve_measure(a.serve_seconds)
    line = {"metric": "served solves/s with p50/p99 latency (Poisson 200 req/s)",
            "value": m["served_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": m["requests"], "warmup": 16, "ms_per_step": 1e3 / m["served_solves_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": "serve", **m["requests_mix"]},
            "serve": m}
    print(json.dumps(line), flush=True)


def run_configs(a):
    """The per-configuration measurements behind the headline: evals/s of each
    evaluation path at the Table 1 sizes (with the oracle's rate on a bounded
    sample), the n = 5000 density-0.1 solve over lambda, the n = 100 small-case
    solve latency, and a multi-round search history (Fig. 3/4-style curve on a
    synthetic ORLIB-shaped instance).  CUDA-event times, L2 flushed before
    every timed call."""
    import torch
    from paper_1706_00037_gb300 import synth, ubqp
    import oracle as orc
    orc.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps, warm=2):
        ts = []
        for r in range(warm + reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(r)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= warm:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16_peak = float(peaks.get("bf16_tflops", 1858.6))
    paper_gpu_s = {2500: 0.7, 5000: 2.0, 6000: 3.0, 7000: 3.5}  # Table 1, 1000 evals
    table1 = {}
    for n in (2500, 5000, 6000, 7000):
        Qh = synth.make_instance(n, 1.0, n)
        inst = ubqp.Instance(torch.from_numpy(Qh).to(dev))
        S = 1000
        X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=n + 1)
        f = torch.empty(S, dtype=torch.int64, device=dev)
        row = {}
        ref = None
        for name, path in (("auto", ubqp.EVAL_AUTO), ("tc_fused", ubqp.EVAL_TC),
                           ("tc_staged", ubqp.EVAL_TC_STAGED), ("plain", ubqp.EVAL_PLAIN)):
            ws = torch.empty(max(ubqp.eval_workspace_size(inst, S, path), 16),
                             dtype=torch.uint8, device=dev)
            ms = timed(lambda r: ubqp.eval(inst, X, path=path, out=f, ws=ws), 10)
            if ref is None:
                ref = f.clone()
            assert torch.equal(f, ref), "evaluation paths disagree"
            row[name] = {"ms_per_1000": ms, "evals_per_s": S / (ms / 1e3),
                         "tflops": S * n * (n + 1) / (ms / 1e3) / 1e12}
            if path != ubqp.EVAL_PLAIN:
                row[name]["frac_of_bf16_burst"] = row[name]["tflops"] / bf16_peak
        inst.sync()
        # the oracle's rate on a bounded sample of the same starts
        Xh = X[:8].cpu().numpy().view(np.uint64)
        t0 = time.perf_counter()
        fh = orc.eval(Qh, Xh)
        dt = time.perf_counter() - t0
        assert np.array_equal(fh, ref[:8].cpu().numpy())
        row["oracle_1core"] = {"evals_per_s": 8 / dt, "sample": "8 starts"}
        if not a.no_cpu:
            Xa = X[:256].cpu().numpy().view(np.uint64)
            fa, dta, procs = oracle_eval_all_cores(n, 1.0, n, Xa)
            assert np.array_equal(fa, ref[:256].cpu().numpy())
            row["oracle_all_cores"] = {"evals_per_s": 256 / dta, "processes": procs,
                                       "sample": "256 starts split over the processes"}
        row["paper_gtx780ti_evals_per_s"] = 1000 / paper_gpu_s[n]
        table1[n] = row
        del inst

    # n = 5000, density 0.1, 8192 DIVERSIFY starts, lambda sweep
    Qh = synth.make_instance(5000, 0.1, 3)
    inst = ubqp.Instance(torch.from_numpy(Qh).to(dev))
    c3 = {}
    for lam in (0.25, 0.5, 0.75):
        params = ubqp.make_params(8192, lam, mode=ubqp.DIVERSIFY, seed=3)
        ws = torch.empty(ubqp.solve_workspace_size(inst, params), dtype=torch.uint8, device=dev)
        bx = torch.empty(inst.words, dtype=torch.int64, device=dev)
        bf = torch.empty(2, dtype=torch.int64, device=dev)
        ms = timed(lambda r: ubqp.solve(inst, params, ws=ws, best_x=bx, best_f=bf,
                                        want_stats=False), 10)
        _, bfv, st = ubqp.solve(inst, params, ws=ws)
        c3[str(lam)] = {"solve_ms": ms, "evals_per_s": 8192 / (ms / 1e3),
                        "passed": st["passed"], "flips": st["total_flips"],
                        "moves_per_s": st["total_flips"] / (ms / 1e3),
                        "best_f": int(bfv[0].item())}
    inst.sync()
    del inst

    # n = 100 small case: latency of one whole solve (1000 DIVERSIFY starts)
    Qh = synth.make_instance(100, 0.1, 0)
    inst = ubqp.Instance(torch.from_numpy(Qh).to(dev))
    params = ubqp.make_params(1000, 0.5, mode=ubqp.DIVERSIFY, seed=0)
    ws = torch.empty(ubqp.solve_workspace_size(inst, params), dtype=torch.uint8, device=dev)
    bx = torch.empty(inst.words, dtype=torch.int64, device=dev)
    bf = torch.empty(2, dtype=torch.int64, device=dev)
    ms = timed(lambda r: ubqp.solve(inst, params, ws=ws, best_x=bx, best_f=bf,
                                    want_stats=False), 20)
    ref = orc.solve(Qh, 1000, 0.5, 0, 0, orc.DIVERSIFY)
    assert int(bf[0].item()) == ref["best_f"]
    # the same round as a one-instance batch plan replayed from its CUDA graph
    # (one launch from the host instead of one per kernel)
    b1 = ubqp.Batch([inst], params)
    b1.tune()
    b1.capture()
    ms_graph = timed(lambda r: b1.run(0), 20)
    _, bfg = b1.result(0)
    assert int(bfg[0].item()) == ref["best_f"]
    b1.close()
    c1 = {"solve_us": ms * 1e3, "evals_per_s": 1000 / (ms / 1e3), "best_f": ref["best_f"],
          "graph_batch_us": ms_graph * 1e3, "equals_oracle": True}
    inst.sync()
    del inst

    # multi-round search on an ORLIB-shaped instance (n = 2500, density 0.1)
    Qh = synth.make_instance(2500, 0.1, 25)
    inst = ubqp.Instance(torch.from_numpy(Qh).to(dev))
    rounds = 40
    res = {}
    ms = timed(lambda r: res.update(ubqp.search(inst, 1000, 1000, rounds, 0.5, seed=25)), 3,
               warm=1)
    hist = res["history"].cpu().tolist()
    search = {"n": 2500, "density": 0.1, "starts_per_round": 1000, "rounds": rounds,
              "num_samples": 1000, "lambda": 0.5, "ms_total": ms, "ms_per_round": ms / rounds,
              "history": hist}
    inst.sync()

    # path relinking (intensification) between elite solutions: the ascended
    # passers of one 1000-start batch, each relinked toward the next one
    relink = {}
    for n in (2500, 7000):
        Qh = synth.make_instance(n, 1.0, n)
        inst = ubqp.Instance(torch.from_numpy(Qh).to(dev))
        S = 1000
        X = ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=77)
        f = ubqp.eval(inst, X)
        idx = torch.arange(S, dtype=torch.int32, device=dev)
        cnt = torch.full((1,), S, dtype=torch.int64, device=dev)
        ubqp.ascent(inst, X, f, idx, cnt)  # 1000 local optima
        order = torch.argsort(f, descending=True)[:256]
        Xe, fe = X[order].contiguous(), f[order].contiguous()
        Ge = torch.roll(Xe, 1, 0).contiguous()
        ws = torch.empty(ubqp.relink_workspace_size(inst, 256), dtype=torch.uint8, device=dev)
        out = {}
        ms = timed(lambda r: out.update(zip(("x", "f", "d"),
                                            ubqp.relink(inst, Xe, fe, Ge, ws=ws))), 10)
        steps = int(out["d"].sum().item())
        Xh, Gh = Xe[:2].cpu().numpy().view(np.uint64), Ge[:2].cpu().numpy().view(np.uint64)
        t0 = time.perf_counter()
        for p in range(2):
            ex, ef, ed = orc.relink1(Qh, Xh[p], Gh[p])
            assert ef == int(out["f"][p].item()) and ed == int(out["d"][p].item())
        dt = time.perf_counter() - t0
        relink[n] = {"pairs": 256, "ms": ms, "pairs_per_s": 256 / (ms / 1e3),
                     "moves_per_s": steps / (ms / 1e3), "mean_distance": steps / 256,
                     "improved_pairs": int((out["f"] > torch.maximum(fe, fe.roll(1, 0)))
                                           .sum().item()),
                     "oracle_1core_pairs_per_s": 2 / dt}
        inst.sync()
        del inst

    line = {"metric": "per-configuration measurements (Table 1 sizes, n=5000 lambda sweep, "
                      "n=100 latency, search history, path relinking)",
            "value": table1[7000]["auto"]["evals_per_s"], "unit": "evals/s (eval only, n=7000)",
            "n_gpus": 1, "steps": 10, "warmup": 2, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "configs", "l2": "flushed before every timed call"},
            "table1": table1, "n5000_d0.1_S8192": c3, "n100_solve": c1, "search": search,
            "relink": relink}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch64":
        return run_batch64(a)
    if a.workload == "serve":
        a.serve_seconds = a.serve_seconds or 60.0
        return run_serve(a)
    if a.workload == "configs":
        return run_configs(a)

    import torch
    import torch.distributed as dist
    from paper_1706_00037_gb300 import synth, ubqp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    path = {"auto": ubqp.EVAL_AUTO, "tc": ubqp.EVAL_TC, "plain": ubqp.EVAL_PLAIN}[a.eval_path]

    n, S = a.n, a.starts
    Qh = synth.make_instance(n, a.density, n)
    Qd = torch.from_numpy(Qh).to(dev)
    inst = ubqp.Instance(Qd)
    W = inst.words
    stream = torch.cuda.current_stream()

    X = torch.empty((S, W), dtype=torch.int64, device=dev)
    f = torch.empty(S, dtype=torch.int64, device=dev)
    idx = torch.empty(S, dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int64, device=dev)
    Tm = torch.empty(2, dtype=torch.float64, device=dev)
    sst = torch.empty(3, dtype=torch.int64, device=dev)
    bx = torch.empty(W, dtype=torch.int64, device=dev)
    bf = torch.empty(2, dtype=torch.int64, device=dev)
    ews = ubqp.eval_workspace_size(inst, S, path)
    aws = ubqp.ascent_workspace_size(inst, S)
    ws = torch.empty(max(ews, aws, 16), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    total_steps = a.warmup + a.steps
    flips_all = torch.zeros((total_steps, S), dtype=torch.int32, device=dev)
    names = ["diversify", "eval", "screen", "ascent", "best"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
           for _ in range(total_steps)]
    lib = ubqp.load()
    sp = ubqp._stream(stream)
    import ctypes
    P = ctypes.c_void_p

    def step(k):
        seed = 1_000_003 * (rank + 1) + k
        e = evs[k]
        e[0].record(stream)
        ubqp._check(lib.ubqp_diversify(inst.handle, None, ubqp.RANDOM, seed, 0, S, 64,
                                       P(X.data_ptr()), sp))
        e[1].record(stream)
        ubqp._check(lib.ubqp_eval(inst.handle, P(X.data_ptr()), S, P(f.data_ptr()), path,
                                  P(ws.data_ptr()), ws.numel(), sp))
        e[2].record(stream)
        ubqp._check(lib.ubqp_screen(P(f.data_ptr()), S, a.lam, P(idx.data_ptr()),
                                    P(count.data_ptr()), P(Tm.data_ptr()), P(sst.data_ptr()),
                                    sp))
        e[3].record(stream)
        ubqp._check(lib.ubqp_ascent(inst.handle, P(X.data_ptr()), P(f.data_ptr()),
                                    P(idx.data_ptr()), P(count.data_ptr()), S, 0,
                                    P(flips_all[k].data_ptr()), P(ws.data_ptr()), ws.numel(),
                                    sp))
        e[4].record(stream)
        ubqp._check(lib.ubqp_best(P(f.data_ptr()), P(X.data_ptr()), S, W, P(bx.data_ptr()),
                                  P(bf.data_ptr()), sp))
        e[5].record(stream)

    for k in range(a.warmup):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    inst.sync()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t_wall = time.perf_counter()
        for k in range(a.warmup, total_steps):
            flush.zero_()
            step(k)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    inst.sync()
    per = np.zeros((a.steps, len(names)))
    for i, k in enumerate(range(a.warmup, total_steps)):
        for j in range(len(names)):
            per[i, j] = evs[k][j].elapsed_time(evs[k][j + 1])
    step_ms = per.sum(axis=1)
    my_total = float(step_ms.sum())
    flips_timed = int(flips_all[a.warmup:].sum().item())
    if world > 1:
        t = torch.tensor([my_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_total = float(t.item())
        fl = torch.tensor([flips_timed], dtype=torch.int64, device=dev)
        dist.all_reduce(fl)
        flips_all_ranks = int(fl.item())
    else:
        max_total, flips_all_ranks = my_total, flips_timed
    clocks = clk.summary()

    value = world * S * a.steps / (max_total / 1e3)
    kern_ms = per.mean(axis=0)
    kernels = {nm: {"ms_per_launch": float(kern_ms[j]),
                    "share": float(kern_ms[j] / kern_ms.sum())} for j, nm in enumerate(names)}
    asc_s = per[:, 3].sum() / 1e3
    moves_per_s = flips_timed / asc_s if asc_s > 0 else None

    # ---- 1-flip moves/s with every start of a batch ascended (no screen):
    # the throughput form of the ascent, two fresh batches, untimed warm-up one.
    all_idx = torch.arange(S, dtype=torch.int32, device=dev)
    all_cnt = torch.full((1,), S, dtype=torch.int64, device=dev)
    flips_a = torch.zeros(S, dtype=torch.int32, device=dev)
    asc_all_ms, asc_all_flips = 0.0, 0
    for rep in range(3):
        ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=777 + rep, out=X)
        ubqp.eval(inst, X, path=path, out=f, ws=ws if ews else None)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ubqp.ascent(inst, X, f, all_idx, all_cnt, 0, flips_a, ws=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            asc_all_ms += e0.elapsed_time(e1)
            asc_all_flips += int(flips_a.sum().item())
    inst.sync()
    moves_all = asc_all_flips / (asc_all_ms / 1e3)

    # ---- several independent rounds in flight (ubqp_solve_rounds): one round's
    # ~50 passers leave most SMs idle during the climb; R rounds of the same
    # workload (1000 random starts each, each screened on its own) share one
    # evaluation and one climb launch.  L2 flushed before every call.
    rounds = {}
    for R in (1, 2, 3, 4):
        rp = ubqp.make_params(S, a.lam, mode=ubqp.RANDOM, seed=31_000 + 10 * R, eval_path=path)
        rws = torch.empty(ubqp.solve_rounds_workspace_size(inst, rp, R), dtype=torch.uint8,
                          device=dev)
        rbx = torch.empty((R, W), dtype=torch.int64, device=dev)
        rbf = torch.empty((R, 2), dtype=torch.int64, device=dev)
        ts = []
        for rep in range(7):
            flush.zero_()
            rp.seed = 31_000 + 10 * R + 1000 * rep
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ubqp.solve_rounds(inst, rp, R, ws=rws, best_x=rbx, best_f=rbf)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep >= 2:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        rounds[str(R)] = {"ms_per_call": ms, "starts_per_s": R * S / (ms / 1e3)}
    inst.sync()

    # ---- roofline of the dominant kernel (ascent).  Per move the ascent reads
    # one int8 row of Q (n bytes, L2-resident) and does 3n integer operations
    # (each element's gain update, key and comparison), so its moves/s are
    # bounded by min(L2 read rate / n, integer rate / 3n); both rates are
    # measured here on this GPU (ubqp_peak_*).  The passers of the timed steps
    # are recounted untimed for the report.
    passers = 0
    for k in range(a.warmup, total_steps):
        seed = 1_000_003 * (rank + 1) + k
        ubqp.diversify(inst, S, mode=ubqp.RANDOM, seed=seed, out=X)
        ubqp.eval(inst, X, path=path, out=f, ws=ws if ews else None)
        sc = ubqp.screen(f, a.lam)
        passers += int(sc["count"].item())
    mp = ubqp.measure_peaks()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = mp["ascent_update_tops"] * 1e12            # ops/s, 3 per element update
    l2_peak = mp["l2_read_gbs"] * 1e9                      # bytes/s
    moves_roof = min(l2_peak / n, alu_peak / (3 * n))
    l2_bound = l2_peak / n < alu_peak / (3 * n)

    def ascent_roofline(moves, secs):
        r = {"kernel": "ascent", "bound": "l2" if l2_bound else "alu",
             "moves_per_s": moves / secs if secs > 0 else None,
             "roofline_moves_per_s": moves_roof}
        if l2_bound:
            r.update(achieved=n * moves / secs / 1e9 if secs > 0 else None,
                     peak=l2_peak / 1e9, unit="GB/s (L2 read)")
        else:
            r.update(achieved=3 * n * moves / secs / 1e12 if secs > 0 else None,
                     peak=alu_peak / 1e12, unit="Tops/s (int32)")
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None
        r["peak_source"] = ("measured in this run on this GPU: the ascent's element update "
                            "(dp4a + multiply-add + three-way max, 3 ops per element) at full "
                            "occupancy" if not l2_bound else
                            "measured in this run on this GPU: 16-byte L2 reads of a "
                            f"{mp['l2_buffer_bytes'] >> 20} MiB resident buffer")
        r["work"] = f"{'n bytes' if l2_bound else '3n int32 ops'} per move, n = {n}"
        return r

    roof_asc = ascent_roofline(flips_timed, asc_s)
    roof_asc["traffic"] = (profiled_traffic("ascent_block_n7000_dense.md",
                                            "traffic_bytes_per_launch") if n == 7000 else None)
    roof_asc_all = ascent_roofline(asc_all_flips, asc_all_ms / 1e3)
    eval_s = per[:, 1].sum() / 1e3
    eval_flops = float(S) * n * (n + 1) * a.steps  # 2 * S * n(n+1)/2 triangle MACs
    tc = ubqp.EVAL_TC if path == ubqp.EVAL_AUTO else path
    if tc == ubqp.EVAL_TC:
        roof_eval = {"kernel": "eval", "bound": "tensor",
                     "achieved": eval_flops / eval_s / 1e12, "unit": "TFLOP/s",
                     "peak": float(peaks.get("bf16_tflops", 1858.6)),
                     "peak_source": "MEASURED_PEAKS bf16_tflops (burst), of measured"}
    else:
        roof_eval = {"kernel": "eval", "bound": "alu",
                     "achieved": eval_flops / 2 / eval_s / 1e12, "unit": "Tops/s (int32)",
                     "peak": n_sm * 128 * sm_max * 1e6 * 4 / 1e12,
                     "peak_source": "derived: dp4a, 4 MACs per int32 lane-op x "
                                    f"{n_sm} SMs x 128 lanes x {sm_max:.0f} MHz"}
    roof_eval["frac"] = roof_eval["achieved"] / roof_eval["peak"]
    if tc == ubqp.EVAL_TC:
        # the operand tiles the tensor-core evaluation moves from L2 into shared
        # memory: per K step of 64, a 128 x 64 bf16 A tile and a 256 x 64 B tile,
        # for every m-tile of 128 starts and every 256-column block J over its
        # K range [0, 256 (J + 1)) (chunks of at most 16 steps)
        n_tc = (n + 255) // 256 * 256
        k_steps = ((S + 127) // 128) * sum(min(4 * (J + 1), n_tc // 64)
                                           for J in range(n_tc // 256))
        tile_bytes = k_steps * (128 + 256) * 64 * 2
        roof_eval["l2_leg"] = {"tile_bytes_per_launch": tile_bytes,
                               "achieved_gbs": tile_bytes * a.steps / eval_s / 1e9,
                               "peak_gbs": mp["l2_read_gbs"],
                               "frac": tile_bytes * a.steps / eval_s / 1e9 / mp["l2_read_gbs"],
                               "peak_source": "measured in this run: L2 read rate"}
    roof_eval["traffic"] = (profiled_traffic("eval_tc_n7000_dense.md",
                                             "traffic_bytes_per_launch_eval")
                            if n == 7000 and tc == ubqp.EVAL_TC else None)
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_launch"])
    roofline = roof_asc if dom == "ascent" else dict(roof_eval)

    # ---- end to end through the public API with host buffers: H2D of the
    # instance, prepare, solve, D2H of the result, every step.
    e2e = None
    if not a.no_e2e:
        Qpin = torch.from_numpy(Qh).pin_memory()
        params = ubqp.make_params(S, a.lam, mode=ubqp.RANDOM, seed=5, eval_path=path)
        out_x = [torch.empty(W, dtype=torch.int64).pin_memory() for _ in range(2)]
        out_f = [torch.empty(2, dtype=torch.int64).pin_memory() for _ in range(2)]
        Qdev = torch.empty_like(Qd)  # staging buffer of the copied Q
        arenas = [torch.empty(ubqp.arena_size(n), dtype=torch.uint8, device=dev)
                  for _ in range(2)]
        wsz = None
        main = torch.cuda.current_stream()
        copy_stream, prep_stream = torch.cuda.Stream(), torch.cuda.Stream()
        done_stream = torch.cuda.Stream()
        ev_copied = torch.cuda.Event()
        ev_prepared = [torch.cuda.Event(), torch.cuda.Event()]
        ev_solved = [torch.cuda.Event(), torch.cuda.Event()]

        def prepare(k, first):
            # step k's Q: copied from pinned host memory into the staging
            # buffer once the previous preparation has read it, then prepared
            # into arena k % 2 once the solve two steps back is done; both on
            # side streams, nothing waits on the host
            b = k & 1
            if k > first:
                copy_stream.wait_event(ev_prepared[(k - 1) & 1])
            with torch.cuda.stream(copy_stream):
                Qdev.copy_(Qpin, non_blocking=True)
            ev_copied.record(copy_stream)
            prep_stream.wait_event(ev_copied)
            if k - 2 >= first:
                prep_stream.wait_event(ev_solved[b])
            inst = ubqp.Instance(Qdev, stream=prep_stream, arena=arenas[b],
                                 defer_validation=True)
            ev_prepared[b].record(prep_stream)
            return inst

        def solve(k, inst):
            nonlocal wsz
            b = k & 1
            main.wait_event(ev_prepared[b])
            params.seed = 77 + k
            need = ubqp.solve_workspace_size(inst, params)
            if wsz is None or wsz.numel() < need:
                wsz = torch.empty(need, dtype=torch.uint8, device=dev)
            bx2, bf2, _ = ubqp.solve(inst, params, ws=wsz, want_stats=False)
            out_x[b].copy_(bx2, non_blocking=True)
            out_f[b].copy_(bf2, non_blocking=True)
            ev_solved[b].record(main)

        def finish(k, inst):
            # step k's result is on the host once that step alone is done (the
            # next step is already queued behind it); then its validation and
            # errors, and the handle is released before its arena is reused
            done_stream.wait_event(ev_solved[k & 1])
            inst.sync(done_stream)
            results.append(int(out_f[k & 1][0]))
            inst.close()

        results = []

        def run(first, count):
            inst, prev = prepare(first, first), None
            for k in range(first, first + count):
                solve(k, inst)
                if prev is not None:
                    finish(k - 1, prev)
                nxt = prepare(k + 1, first) if k + 1 < first + count else None
                prev, inst = inst, nxt
            finish(first + count - 1, prev)

        ke = max(2, min(a.steps, 50))
        run(0, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(100, ke)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": world * S * ke / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(Qh.nbytes),
               "d2h_bytes_per_step": int(out_x[0].numel() * 8 + out_f[0].numel() * 8),
               "what": "per step: instance Q copied from pinned host memory and "
                       "prepared into one of two arenas (ubqp_q_prepare_into_async) on "
                       "side streams, overlapping the previous step's solve (the first "
                       "step's are not overlapped); ubqp_solve; best solution and value "
                       "back to host; ubqp_sync on a stream ordered after that step alone "
                       "(the next step already queued) reports its validation and errors"}

    served = None
    if rank == 0 and world == 1 and not a.no_serve:
        served = serve_measure(a.serve_seconds or 60.0)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        import oracle as orc
        orc.build()
        op = OraclePool(n, a.density, n)
        try:
            S_cpu = a.cpu_sample * op.procs
            dt, _ = cpu_sample_all_cores(op, a, S_cpu, 4242)
        finally:
            op.close()
        S_one = a.cpu_sample
        dt1, _ = cpu_sample(a, Qh, S_one, 4242)
        cpu = {"value": S_cpu / dt, "unit": UNIT, "cores": op.procs, "kind": "oracle",
               "sample": f"{S_cpu} random starts of the same instance through the whole "
                         f"path (eval, screen over the batch, ascent of passers, best), "
                         f"spread over {op.procs} processes (one per host core), "
                         f"{dt:.1f} s",
               "single_thread": {"value": S_one / dt1, "cores": 1,
                                 "sample": f"{S_one} starts, {dt1:.1f} s"}}

    if rank == 0:
        # diversify 1, eval 1 (fused or plain) or 2 (unpack + tensor-core, staged),
        # screen 1, ascent 3 or 4 (unpack + tensor-core start-up + the climb, and
        # for more listed starts than its blocks hold at once the count-gated
        # throughput twin), best 1
        n_tc = (n + 255) // 256 * 256
        staged = path == ubqp.EVAL_TC_STAGED or (path == ubqp.EVAL_AUTO and not (n_tc <= 1024 and S >= 4096))
        cap = 152 if n > 4096 else (304 if n > 2048 else 456)
        twin = 1024 < n <= 8192 and S > cap
        launches_per_step = 1 + (2 if staged else 1) + 1 + (4 if twin else 3) + 1
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": max_total / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "config": config_of(a, world),
                "moves_per_s": moves_per_s * world if moves_per_s else None,
                "moves_per_s_all_starts_ascended": moves_all * world,
                "ascent_all_starts_ms": asc_all_ms / 2,
                "eval_only_evals_per_s": S * a.steps / eval_s,
                "paper_table1_context": {"evals_per_s_n7000_gtx780ti": 1000 / 3.5},
                "passed_per_step": passers / a.steps, "flips_per_step": flips_timed / a.steps,
                "kernels": kernels, "roofline": roofline, "roofline_eval": roof_eval,
                "roofline_ascent_all_starts": roof_asc_all,
                "rounds_in_flight": {"what": "ubqp_solve_rounds: R independent rounds of the "
                                             "same workload (1000 random starts each, each "
                                             "screened on its own), one evaluation and one "
                                             "climb launch; bit-identical to R ubqp_solve calls",
                                     "by_R": rounds},
                "measured_peaks": dict(mp, sm_max_mhz=sm_max,
                                       int32_lane_peak_tops=n_sm * 128 * sm_max * 1e6 / 1e12),
                "cpu_baseline": cpu, "e2e": e2e,
                "served": served,
                "clocks": clocks, "gpu_launches": launches_per_step * a.steps,
                "wall_s_timed_region": t_wall}
        print(json.dumps(line), flush=True)
    inst.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
