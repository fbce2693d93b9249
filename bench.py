#!/usr/bin/env python
"""Throughput of CTD-S (Algorithm 1 end to end: norms, CDF, sampling,
unique, gather, Gram + in-order filter, U, C = R^T X and the relative error)
on the 10^4 x 10^4 x 10^3 traffic tensor with 10^7 nonzeros (Zipf(1.2)
source/destination ids, uniform time, Geometric(0.3) counts), s = 500,
eps = 1e-6, FP32 bulk storage of C with FP64 U/filter/error.

One JSON line on rank 0.  `value` = nonzeros decomposed per second over all
ranks (each rank decomposes its own tensor: weak scaling, no collective in
the data path), device-timed with CUDA events on the library's stream.
`--impl reference` times the FP64 CPU oracle instead (bounded samples).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NNZ_FULL = 10_000_000
S, EPS = 500, 1e-6
ORACLE_SCALE = 0.3          # bounded CPU sample: 3,000 x 3,000 x 300, 270K nonzeros
WORKLOAD = "CTD-S traffic tensor 10000x10000x1000, 1e7 nnz, Zipf(1.2) src/dst, Geometric(0.3)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink every mode (and nnz by scale^3) for profiling runs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default launch shapes instead of the autotuned ones")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the small-tensor latency, batched and serving measurements")
    return ap.parse_args()


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Each rank decomposes its own replica of the workload with its own
    sampling seed (weak scaling: the units are independent problems)."""
    return rank


def max_over_ranks(ms: float, world: int, device="cpu") -> float:
    """The slowest rank's time; the whole job's value is counted against it."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as td
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(nnz_per_rank: int, world: int, ms_max: float) -> float:
    """Nonzeros decomposed by all ranks per second of the slowest rank."""
    return nnz_per_rank * world / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start sampling: wait for its first line
        # (up to 3 s) so that the samples cover the whole timed region
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel_src: str):
    """DRAM bytes of one C fill (its three kernels) from the committed ncu
    summary, scaled to the full workload; valid only while the kernels'
    source file is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if rec.get("source_sha") == h:
            return rec
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, %r)
from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
coo = synth.traffic_10m(scale=%r)
t0 = time.perf_counter()
ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, %d, %r, 0)
C = O.c_full(ref.X, ref.R)
e = O.projection_error(ref.X, ref.R)
dt = time.perf_counter() - t0
print(json.dumps({"nnz": int(coo.nnz), "seconds": dt, "err": e, "dims": list(coo.dims)}))
"""


def run_oracle_sample():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET % (ROOT, ORACLE_SCALE, S, EPS)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_desc(r):
    d = r["dims"]
    return (f"oracle (numpy FP64, literal Algorithm 1 + exact C + Lemma 3.2 error) on the same "
            f"generator at scale {ORACLE_SCALE}: {d[0]}x{d[1]}x{d[2]}, {r['nnz']} nonzeros, s={S}")


def reference_arm(args):
    rank, world, _ = dist()
    if rank != 0:
        return
    for _ in range(args.warmup):
        run_oracle_sample()
    tot_s, tot_nnz, last = 0.0, 0, None
    for _ in range(args.steps):
        r = run_oracle_sample()
        tot_s += r["seconds"]
        tot_nnz += r["nnz"]
        last = r
    v = tot_nnz / tot_s
    line = {"impl": "reference", "metric": "CTD-S nonzeros/s", "value": v, "unit": "nnz/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample_desc(last)},
            "cpu_baseline": {"value": v, "unit": "nnz/s", "cores": 1, "kind": "oracle",
                             "sample": sample_desc(last)},
            "e2e": {"value": v, "unit": "nnz/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads, measured after the headline (outside its timed region)
# ---------------------------------------------------------------------------
def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=float), q))


def small_latency(ctd, synth, st, gpu):
    """CTD-S on the 100 x 100 x 50 tensor (5,000 uniform nonzeros, Poisson(3)+1,
    s = 50, FP64): wall time of one call through the C ABI with the error
    read back, device-resident input."""
    import torch
    X = ctd.Coo.from_synth(synth.small_uniform())
    for _ in range(5):
        ctd.ctd_static(X, 1, 50, EPS, 0, ctd.CTD_FP64, 0, st).free()
    clocks = ClockSampler(gpu)
    clocks.start()
    ts = []
    for _ in range(200):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F = ctd.ctd_static(X, 1, 50, EPS, 0, ctd.CTD_FP64, 0, st)
        F.error()
        ts.append((time.perf_counter() - t0) * 1e6)
        F.free()
    clocks.stop()
    return {"workload": "CTD-S 100x100x50, 5,000 uniform nonzeros, Poisson(3)+1, s = 50, FP64",
            "calls": len(ts), "p50_us": percentile(ts, 50), "p99_us": percentile(ts, 99),
            "clocks": clocks.summary()}


def stream_form(ctd, synth, gpu, steps=6):
    """The first `steps` of the CTD-D stream of 20,000 x 20,000 slices (5*10^5
    Zipf(1.1) nonzeros each, Poisson(2)+1 counts, d = 400, FP32 bulk): device
    time of each step (synchronized on both sides), slices built on the host
    before it.  The early steps are the cheap ones: the basis is still
    small; the whole 100-step stream is measured by `measure.py stream`."""
    import torch
    st = synth.traffic_stream_20k(scale=1.0, steps=100)
    G = ctd.Dynamic(st.dims2, 1, ctd.CTD_FP32_BULK, 0, 0, ctd.CTD_KEEP_LAST_C)
    clocks = ClockSampler(gpu)
    per, tot_nnz, tot_s = [], 0, 0.0
    slices = [st.slice(t) for t in range(steps)]
    clocks.start()
    for t, sl in enumerate(slices):
        X = ctd.Coo.from_synth(sl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.step_slice(X, 400, EPS)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        per.append(round(dt * 1e3, 3))
        tot_nnz += sl.nnz
        tot_s += dt
    clocks.stop()
    out = {"workload": f"first {steps} of 100 CTD-D steps, 20000x20000 slices, "
                       f"{st.nnz} nonzeros each, d = 400, FP32 bulk",
           "nnz_per_s": tot_nnz / tot_s, "ms_per_step": per, "d_kept": int(G.sizes().s_kept),
           "rel_error": G.error(), "clocks": clocks.summary()}
    G.free()
    return out


def batched_form(ctd, synth, gpu):
    """The 256-tensor law (I, J log-uniform in [500, 2*10^4], K in [10, 500],
    nnz log-uniform in [10^4, 2*10^6], Zipf(1.2) ids, Poisson(3)+1 counts,
    s = min(I, J) / 20), drawn on the device: a plain loop of ctd_static
    against one ctd_static_batched call, same seeds, FP32 bulk; the worker
    count is autotuned on a sample of the tensors first."""
    import torch
    from paper_1710_03608_gb300 import measure
    specs = synth.batch_256()
    t0 = time.perf_counter()
    Xs = [ctd.Coo(sp.dims, *synth.traffic_device(sp.dims, sp.nnz, 1.2, 1.2, "poisson1", 3.0,
                                                 sp.seed)) for sp in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    s = [sp.s for sp in specs]
    seeds = list(range(len(specs)))
    nnz = sum(sp.nnz for sp in specs)
    sample = list(range(0, len(Xs), 8))
    tune = measure.autotune_workers([Xs[i] for i in sample], [s[i] for i in sample],
                                    [seeds[i] for i in sample], candidates=(4, 8, 16),
                                    save=False)
    workers = tune["best"]
    for X, si, se in zip(Xs[:4], s[:4], seeds[:4]):
        ctd.ctd_static(X, 1, si, EPS, se, ctd.CTD_FP32_BULK).free()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu)
    clocks.start()
    t0 = time.perf_counter()
    errs_plain = []
    for X, si, se in zip(Xs, s, seeds):
        F = ctd.ctd_static(X, 1, si, EPS, se, ctd.CTD_FP32_BULK)
        errs_plain.append(F.error())
        F.free()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    Fs = ctd.ctd_static_batched(Xs, 1, s, seeds, EPS, ctd.CTD_FP32_BULK, 0, workers)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    clocks.stop()
    errs_batch = [F.error() for F in Fs]
    # the stated FP32-bulk bar on the error: 1e-4 relative, 1e-6 absolute below 1e-8
    bar = [1e-6 if b < 1e-8 else 1e-4 * b for b in errs_plain]
    same = all(abs(a - b) <= t for a, b, t in zip(errs_batch, errs_plain, bar))
    worst_abs = max(abs(a - b) for a, b in zip(errs_plain, errs_batch))
    return {"workload": f"{len(specs)} uneven CTD-S traffic tensors, {nnz} nonzeros, drawn on "
                        "the device (same law as the 256-tensor workload)",
            "nnz": nnz, "generation_s": gen_s,
            "plain": {"seconds": t_plain, "nnz_per_s": nnz / t_plain},
            "batched": {"seconds": t_batch, "nnz_per_s": nnz / t_batch, "workers": workers},
            "gain": t_plain / t_batch, "same_accuracy": same, "max_abs_error_difference": worst_abs,
            "min_error": min(errs_plain), "max_error": max(errs_plain),
            "autotune": tune, "clocks": clocks.summary()}


def serving_form(ctd, synth, gpu, seconds=0.25):
    """64 CTD-D streams with Poisson arrivals at 2 kHz in total for `seconds`
    s, each request one 5,000 x 5,000 slice with nnz log-uniform in
    [10^4, 10^6] (Zipf(1.1) ids, Poisson(3)+1 counts, drawn on the device),
    d = 200, FP32 bulk: continuous batching against one request at a time,
    the same paced arrivals; latency from submission to completion."""
    import numpy as np
    import torch
    from paper_1710_03608_gb300 import measure
    dims = (5000, 5000, 1)
    reqs = synth.serving_requests(streams=64, rate_hz=2000.0, duration_s=seconds)
    Xs = [ctd.Coo(dims, *synth.traffic_device(dims, r.nnz, 1.1, 1.1, "poisson1", 3.0, r.seed))
          for r in reqs]
    torch.cuda.synchronize()
    total = sum(r.nnz for r in reqs)

    def run(workers):
        S = ctd.Server(64, dims[:2], 200, EPS, 1, ctd.CTD_FP32_BULK, 0, workers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for r, X in zip(reqs, Xs):
            while time.perf_counter() - t0 < r.arrival_s:
                time.sleep(0.0001)
            tickets.append(S.submit(r.stream, X))
        S.wait()
        wall = time.perf_counter() - t0
        lat = np.array([S.result(t)[1][2] for t in tickets])
        S.close()
        return wall, lat

    workers = measure.tuned_workers()
    clocks = ClockSampler(gpu)
    clocks.start()
    w_mix, lat_mix = run(workers)
    clocks.stop()
    w_one, lat_one = run(1)
    return {"workload": f"64 CTD-D streams, 5000x5000 slices, Poisson arrivals at 2 kHz for "
                        f"{seconds} s ({len(reqs)} requests, {total} nonzeros), d = 200",
            "offered_nnz_per_s": total / seconds,
            "continuous": {"workers": workers, "achieved_nnz_per_s": total / w_mix,
                           "p50_ms": percentile(lat_mix, 50), "p99_ms": percentile(lat_mix, 99),
                           "wall_s": w_mix},
            "one_at_a_time": {"achieved_nnz_per_s": total / w_one,
                              "p50_ms": percentile(lat_one, 50),
                              "p99_ms": percentile(lat_one, 99), "wall_s": w_one},
            "gain": w_one / w_mix, "clocks": clocks.summary()}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def c_fill_bytes(sz):
    """Algorithmic bytes of one C = R^T X launch by the per-unit figures of the
    method's hot-path table: X read by column (row and value, 8 B per
    nonzero), C written as (row, column, value) triples (12 B per nonzero of
    C) and a 4-byte column offset per column of X_(alpha).  The library's
    layout writes fewer bytes than this (16-bit rows, dense columns without
    row indices); the measured DRAM bytes are `traffic`."""
    return 8 * sz.nnz_X + 12 * sz.nnz_C + 4 * sz.n_cols


def ours(args):
    import numpy as np
    import torch

    from paper_1710_03608_gb300 import ctd, synth
    rank, world, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
    ctd.load()
    coo = synth.traffic_10m(scale=args.scale)
    nnz_step = coo.nnz
    X = ctd.Coo.from_synth(coo)
    st = torch.cuda.current_stream()
    seed = rank_seed(rank)

    def barrier():
        if world > 1:
            import torch.distributed as td
            td.barrier()

    def step(Xd):
        F = ctd.ctd_static(Xd, 1, S, EPS, seed, ctd.CTD_FP32_BULK, 0, st)
        return F

    for _ in range(max(args.warmup, 3)):
        step(X).free()
    torch.cuda.synchronize()
    # the launch-shape autotuner on this workload, before the timed region:
    # the knobs change how the hot kernels are laid out, never what they
    # compute; the timed steps run with the setting it picks
    from paper_1710_03608_gb300 import measure
    tune = None
    if not args.no_autotune:
        tune = measure.autotune_kernels(X, S, seed, save=False)
    sizes = None
    clocks = ClockSampler(local)
    ctd.profile(True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    err = None
    for k in range(args.steps):
        F = step(X)
        if k == args.steps - 1:
            sizes = F.sizes()
            err = F.error()
            last = F
            continue
        F.free()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    clocks.stop()
    from paper_1710_03608_gb300 import measure
    mem_usage = measure.memory_usage(last)   # Eq. (memoryEff), read after the timed region
    last.free()
    ms = e0.elapsed_time(e1) / args.steps
    rep = ctd.profile_report()
    ctd.profile(False)
    t_max = max_over_ranks(ms, world, device="cuda")
    value = whole_job_value(nnz_step, world, t_max)

    # live roofline of the dominant kernel (C = R^T X)
    peak, peak_kind = measured_peaks()
    ph = rep["phases"]
    cf = ph.get("c_fill", {"ms": float("nan"), "calls": 1})
    cf_ms = cf["ms"] / max(cf["calls"], 1)
    alg = c_fill_bytes(sizes)
    achieved = alg / (cf_ms * 1e-3) / 1e9
    tr = ncu_traffic(os.path.join(ROOT, "paper_1710_03608_gb300", "csrc", "ctd_cfill.cu"))
    traffic = tr["bytes_per_launch"] if tr else None
    roof = {"kernel": "C = R^T X_(alpha) (k_img_*, k_copy_flat, k_cf; column lists from the bounds pass)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "algorithmic_bytes": alg, "ms": cf_ms,
            "traffic": traffic,
            # DRAM bytes the launch moved (ncu) over its live duration
            "dram_frac": (traffic / (cf_ms * 1e-3) / 1e9 / peak) if traffic else None}
    # the same fill with nothing beside it: three calls with the error off
    # (CTD_SKIP_ERROR), after the timed region; inside it the error's kernels
    # share the GPU with the fill from a second stream
    ctd.profile(True)
    for _ in range(3):
        ctd.ctd_static(X, 1, S, EPS, seed, ctd.CTD_FP32_BULK, ctd.CTD_SKIP_ERROR, st).free()
    torch.cuda.synchronize()
    ph_alone = ctd.profile_report()["phases"]
    ctd.profile(False)
    cfa = ph_alone.get("c_fill", {"ms": float("nan"), "calls": 1})
    cfa_ms = cfa["ms"] / max(cfa["calls"], 1)
    roof["alone"] = {"ms": cfa_ms, "achieved": alg / (cfa_ms * 1e-3) / 1e9,
                     "frac": alg / (cfa_ms * 1e-3) / 1e9 / peak,
                     "dram_frac": (traffic / (cfa_ms * 1e-3) / 1e9 / peak) if traffic else None,
                     "how": "3 calls with the error off, after the timed region"}
    phases = {k: {"ms_per_step": round(v["ms"] / args.steps, 4),
                  "calls_per_step": round(v["calls"] / args.steps, 2)} for k, v in ph.items()}
    if "call" in ph:
        # device time of a call not covered by a named phase (mostly idle
        # gaps while the host reads back sizes and issues the next kernels)
        # sub-phases (c_fill_copy, c_fill_multi) sit inside c_fill: not counted twice
        inner = sum(v["ms"] for k, v in ph.items() if k != "call" and not k.startswith("c_fill_"))
        phases["between_phases"] = {"ms_per_step": round((ph["call"]["ms"] - inner) / args.steps, 4),
                                    "calls_per_step": 1.0}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pins = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).pin_memory()
                for a in (coo.i, coo.j, coo.k, coo.val)]
        Xh = ctd.Coo(coo.dims, *[p.numpy() for p in pins])
        step(Xh).free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            F = step(Xh)
            _ = F.error()          # device -> host read of the step's result
            F.free()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        e2e = {"value": nnz_step / dt, "unit": "nnz/s", "h2d_bytes_per_step": 16 * coo.nnz,
               "d2h_bytes_per_step": 8, "ms_per_step": dt * 1e3}

    # defaults back for the other workloads
    for k in measure.KNOB_GRID:
        ctd.set_tuning(k, -1)
    extra = {}
    if tune is not None:
        extra["kernel_autotune"] = tune
    if rank == 0 and world == 1 and not args.no_extra and args.scale == 1.0:
        extra["small_tensor_latency"] = small_latency(ctd, synth, st, local)
        try:
            extra["stream"] = stream_form(ctd, synth, local)
        except Exception as e:  # a sample of another config must not cost the line
            extra["stream"] = {"error": f"{type(e).__name__}: {e}"}
        extra["batched"] = batched_form(ctd, synth, local)
        extra["serving"] = serving_form(ctd, synth, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle_sample()
        cpu = {"value": r["nnz"] / r["seconds"], "unit": "nnz/s", "cores": 1, "kind": "oracle",
               "sample": sample_desc(r), "seconds": r["seconds"]}

    if rank == 0:
        line = {"metric": "CTD-S nonzeros/s", "value": value, "unit": "nnz/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.scale == 1.0 else
                           f"{WORKLOAD} at scale {args.scale}: dims {list(coo.dims)}",
                           "s": S, "eps": EPS, "precision": "FP32_BULK", "nnz": nnz_step, "s_unique": sizes.s_unique, "s_kept": sizes.s_kept,
                           "nnz_R": sizes.nnz_R, "nnz_C": sizes.nnz_C, "rel_error": err,
                           "memory_usage": mem_usage,
                           "l2": "inputs larger than L2 (160 MB COO, 5+ GB C per step)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "phases_ms": phases, "gpu_launches": rep["launches"],
                "clocks": clocks.summary(), "e2e": e2e, "cpu_baseline": cpu, **extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
