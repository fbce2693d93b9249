"""Measurements of the batched, serving and streaming forms (one JSON line each).

  python -m paper_1710_03608_gb300.measure batched [--count N] [--tune]
      256 uneven CTD-S tensors: a plain loop of ctd_static vs one
      ctd_static_batched call; nonzeros/s of each and the gain.
  python -m paper_1710_03608_gb300.measure serving [--seconds S] [--rate HZ]
      64 CTD-D streams, Poisson arrivals, continuous batching; p50/p99
      latency, offered and achieved nonzeros/s; the same requests run one at
      a time for comparison.
  python -m paper_1710_03608_gb300.measure stream [--steps T] [--scale F]
      one CTD-D stream of 2*10^4 x 2*10^4 slices (500K nonzeros each, planted
      block at steps 40-45); per-step nonzeros/s and d~_t.
  python -m paper_1710_03608_gb300.measure ncu-summary LAUNCHES.csv
  python -m paper_1710_03608_gb300.measure ncu-dram DRAM.csv --peak GBS
      per-kernel launches, time and share of an ncu launch list (no GPU).

All times are host wall-clock around calls that wait for their work (the
library's entry points return when the device is done), inputs in HBM.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import ctd, synth

_HERE = os.path.dirname(os.path.abspath(__file__))
TUNE_FILE = os.path.join(_HERE, "_build", "autotune.json")


def _sync():
    import torch
    torch.cuda.synchronize()


def memory_usage(F) -> float:
    """Eq. (memoryEff) of the paper's Section 4 for CTD-S factors:
    (nnz(C) + nnz(U) + nnz(R)) / nnz(X), nonzero entries counted; an entry
    of U counts when its magnitude exceeds 1e-12 of U's largest (U is read
    back to count)."""
    sz = F.sizes()
    nnz_u = 0
    if sz.s_kept:
        U = np.abs(F.U())
        nnz_u = int(np.count_nonzero(U > 1e-12 * U.max()))
    return (sz.nnz_C + nnz_u + sz.nnz_R) / max(sz.nnz_X, 1)


# ---------------------------------------------------------------------------
# autotuner: worker streams for the batched form
# ---------------------------------------------------------------------------
def _tune_load() -> dict:
    try:
        with open(TUNE_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


def _tune_save(update: dict) -> None:
    d = _tune_load()
    d.update(update)
    os.makedirs(os.path.dirname(TUNE_FILE), exist_ok=True)
    with open(TUNE_FILE, "w") as f:
        json.dump(d, f)


def tuned_workers(default: int = 8) -> int:
    try:
        return int(_tune_load()["batched_workers"])
    except Exception:
        return default


# ---------------------------------------------------------------------------
# launch-shape autotuner of the hot kernels (ctd_set_tuning knobs)
# ---------------------------------------------------------------------------
KNOB_GRID = {"qform_hot_kb": (0, 100, 150, 200),
             "cfill_dense_kb": (128, 176, 220),
             "copy_blocks_per_sm": (2, 4, 8, 16)}


def size_class(nnz: int) -> str:
    """Workloads are tuned per decade of nonzeros."""
    import math
    return f"nnz_1e{int(round(math.log10(max(int(nnz), 1))))}"


def _time_calls(X, s, seed, calls: int) -> float:
    """Mean device time (ms) of `calls` ctd_static calls, CUDA events on the
    current stream, after one untimed call."""
    import torch
    st = torch.cuda.current_stream()
    ctd.ctd_static(X, 1, s, 1e-6, seed, ctd.CTD_FP32_BULK, 0, st).free()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(calls):
        ctd.ctd_static(X, 1, s, 1e-6, seed, ctd.CTD_FP32_BULK, 0, st).free()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / calls


def autotune_kernels(X, s, seed=0, calls: int = 5, save: bool = True) -> dict:
    """One pass of coordinate descent over the knobs of KNOB_GRID on CTD-S of
    X (FP32_BULK): each knob in turn takes the value with the shortest mean
    call, the others held at their best so far.  The knobs change launch
    shapes only, never results.  The best setting is kept in the tuning
    file under the tensor's size class; the knobs are left at it."""
    best = {k: ctd.get_tuning(k) for k in KNOB_GRID}
    for k, v in best.items():
        ctd.set_tuning(k, v)
    base = _time_calls(X, s, seed, calls)
    sweep = {}
    for k, values in KNOB_GRID.items():
        times = {}
        for v in values:
            ctd.set_tuning(k, v)
            times[v] = min(_time_calls(X, s, seed, calls) for _ in range(2))
        best[k] = min(times, key=times.get)
        ctd.set_tuning(k, best[k])
        sweep[k] = times
    # the default and the tuned setting once more, alternately
    tuned, default = [], []
    for _ in range(2):
        for key in KNOB_GRID:
            ctd.set_tuning(key, -1)
        default.append(_time_calls(X, s, seed, calls))
        for key, v in best.items():
            ctd.set_tuning(key, v)
        tuned.append(_time_calls(X, s, seed, calls))
    cls = size_class(X.desc.nnz)
    if save:
        kern = _tune_load().get("kernels", {})
        kern[cls] = best
        _tune_save({"kernels": kern})
    return {"class": cls, "best": best, "default_ms": min(default), "tuned_ms": min(tuned),
            "first_ms": base, "sweep_ms": sweep, "calls": calls}


def apply_tuning(nnz: int) -> dict:
    """Set the knobs the tuning file holds for nnz's size class (defaults
    when it holds none); returns what was set."""
    best = _tune_load().get("kernels", {}).get(size_class(nnz), {})
    for k in KNOB_GRID:
        ctd.set_tuning(k, best.get(k, -1))
    return {k: ctd.get_tuning(k) for k in KNOB_GRID}


def autotune_workers(Xs, s, seeds, candidates=(2, 4, 8, 12, 16, 24), save: bool = True) -> dict:
    """Time ctd_static_batched on the given tensors for each worker count;
    keep the fastest in the tuning file (when `save`)."""
    times = {}
    for w in candidates:
        for _ in range(2):
            _sync()
            t0 = time.perf_counter()
            Fs = ctd.ctd_static_batched(Xs, 1, s, seeds, 1e-6, ctd.CTD_FP32_BULK, 0, w)
            _sync()
            dt = time.perf_counter() - t0
            del Fs
        times[w] = dt
    best = min(times, key=times.get)
    if save:
        _tune_save({"batched_workers": best, "times_s": times})
    return {"best": best, "times_s": times}


# ---------------------------------------------------------------------------
# batched CTD-S
# ---------------------------------------------------------------------------
def batched(args):
    specs = synth.batch_256(count=args.count)
    t0 = time.perf_counter()
    tensors = [sp.tensor() for sp in specs]
    gen_s = time.perf_counter() - t0
    Xs = [ctd.Coo.from_synth(x) for x in tensors]
    s = [sp.s for sp in specs]
    seeds = list(range(len(specs)))
    nnz = sum(x.nnz for x in tensors)
    tune = None
    if args.tune:
        sample = list(range(0, len(Xs), max(1, len(Xs) // 48)))
        tune = autotune_workers([Xs[i] for i in sample], [s[i] for i in sample],
                                [seeds[i] for i in sample])
    workers = args.workers or tuned_workers()
    # warm-up
    ctd.ctd_static_batched(Xs[:8], 1, s[:8], seeds[:8], 1e-6, ctd.CTD_FP32_BULK, 0, workers)
    for X, si, se in zip(Xs[:4], s[:4], seeds[:4]):
        ctd.ctd_static(X, 1, si, 1e-6, se, ctd.CTD_FP32_BULK)
    _sync()
    # plain loop
    t0 = time.perf_counter()
    errs_plain = []
    for X, si, se in zip(Xs, s, seeds):
        F = ctd.ctd_static(X, 1, si, 1e-6, se, ctd.CTD_FP32_BULK)
        errs_plain.append(F.error())
        F.free()
    _sync()
    t_plain = time.perf_counter() - t0
    # batched
    t0 = time.perf_counter()
    Fs = ctd.ctd_static_batched(Xs, 1, s, seeds, 1e-6, ctd.CTD_FP32_BULK, 0, workers)
    _sync()
    t_batch = time.perf_counter() - t0
    errs_batch = [F.error() for F in Fs]
    # integer stages are bit-exact; the FP32 error sum may differ in its last bits
    same = all(abs(a - b) <= 1e-6 * max(abs(b), 1e-6) for a, b in zip(errs_plain, errs_batch))
    line = {"workload": f"{len(specs)} uneven CTD-S traffic tensors (batch law of the 256-tensor "
                        f"workload), {nnz} nonzeros", "nnz": nnz, "generation_s": gen_s,
            "plain": {"seconds": t_plain, "nnz_per_s": nnz / t_plain},
            "batched": {"seconds": t_batch, "nnz_per_s": nnz / t_batch, "workers": workers},
            "gain": t_plain / t_batch, "same_errors": same, "autotune": tune}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving CTD-D
# ---------------------------------------------------------------------------
def serving(args):
    import torch
    dims2 = (5000, 5000)
    reqs = synth.serving_requests(streams=args.streams, rate_hz=args.rate,
                                  duration_s=args.seconds)
    rng = np.random.default_rng(7)
    # a pool of distinct slices reused cyclically (generation is slower than 2 kHz)
    pool_n = min(args.pool, len(reqs))
    pool = [Request_slice(r, dims2) for r in reqs[:pool_n]]
    Xp = [ctd.Coo.from_synth(sl) for sl in pool]
    nnz = [sl.nnz for sl in pool]
    total_nnz = sum(nnz[q % pool_n] for q in range(len(reqs)))

    def run(workers, paced):
        S = ctd.Server(args.streams, dims2, args.d, 1e-6, 1, ctd.CTD_FP32_BULK, 0, workers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for q, r in enumerate(reqs):
            if paced:
                while time.perf_counter() - t0 < r.arrival_s:
                    time.sleep(0.0002)
            tickets.append(S.submit(r.stream, Xp[q % pool_n]))
        S.wait()
        t_end = time.perf_counter()
        lat = np.array([S.result(t)[1][2] for t in tickets])
        S.close()
        return t_end - t0, lat

    d_mix, lat_mix = run(args.workers, True)
    d_one, lat_one = run(1, True)
    line = {"workload": f"{args.streams} CTD-D streams, 5000x5000 slices, Poisson arrivals at "
                        f"{args.rate:.0f} Hz for {args.seconds} s ({len(reqs)} requests, "
                        f"{pool_n} distinct slices reused), d = {args.d}",
            "offered_nnz_per_s": total_nnz / args.seconds,
            "continuous": {"workers": args.workers, "achieved_nnz_per_s": total_nnz / d_mix,
                           "p50_ms": float(np.percentile(lat_mix, 50)),
                           "p99_ms": float(np.percentile(lat_mix, 99)), "wall_s": d_mix},
            "one_at_a_time": {"achieved_nnz_per_s": total_nnz / d_one,
                              "p50_ms": float(np.percentile(lat_one, 50)),
                              "p99_ms": float(np.percentile(lat_one, 99)), "wall_s": d_one},
            "gain": d_one / d_mix}
    print(json.dumps(line), flush=True)


def Request_slice(r, dims2):
    return r.slice(dims2)


# ---------------------------------------------------------------------------
# one CTD-D stream
# ---------------------------------------------------------------------------
def stream(args):
    st = synth.traffic_stream_20k(scale=args.scale, steps=args.steps)
    G = ctd.Dynamic(st.dims2, 1, ctd.CTD_FP32_BULK, 0, 0, ctd.CTD_KEEP_LAST_C)
    ctd.profile(True)
    per = []
    tot_nnz, tot_s = 0, 0.0
    for t in range(args.steps):
        sl = st.slice(t)
        X = ctd.Coo.from_synth(sl)
        _sync()
        t0 = time.perf_counter()
        G.step_slice(X, args.d, 1e-6)
        _sync()
        dt = time.perf_counter() - t0
        info, sq = G.step(t)
        per.append({"t": t, "nnz": sl.nnz, "ms": dt * 1e3, "d_unique": int(info[0]),
                    "kept": int(info[1]), "d_before": int(info[2])})
        tot_nnz += sl.nnz
        tot_s += dt
    line = {"workload": f"CTD-D stream of {args.steps} slices {st.dims2[0]}x{st.dims2[1]}, "
                        f"{st.nnz} nonzeros each, d = {args.d}",
            "nnz_per_s": tot_nnz / tot_s, "seconds": tot_s, "final_d": int(G.sizes().s_kept),
            "rel_error": G.error(), "phases_ms": ctd.profile_report()["phases"], "steps": per}
    print(json.dumps(line), flush=True)


def ddos(args):
    """Section 5's detector on the C3-shaped stream with its planted block
    (200 sources x 50 destinations of Poisson(40) counts at steps 40-45, the
    block scaled with the slice): CTD-D with the paper's detector setting
    (d = 10, eps = 0.15), the detector run after every step, scored against
    the planted destinations."""
    st = synth.traffic_stream_20k(scale=args.scale, steps=args.steps)
    G = ctd.Dynamic(st.dims2, 1, ctd.CTD_FP32_BULK, 0, 0, ctd.CTD_KEEP_LAST_C)
    truth = set(int(x) for x in st.planted_dst)
    ctd.profile(True)
    step_s, det_s, tot_nnz = 0.0, [], 0
    trace = []
    for t in range(args.steps):
        sl = st.slice(t)
        X = ctd.Coo.from_synth(sl)
        _sync()
        t0 = time.perf_counter()
        G.step_slice(X, args.d, args.eps)
        _sync()
        t1 = time.perf_counter()
        cand, mean = G.ddos_candidates()
        t2 = time.perf_counter()
        step_s += t1 - t0
        det_s.append(t2 - t1)
        tot_nnz += sl.nnz
        hit = len(truth & set(int(x) for x in cand))
        trace.append({"t": t, "candidates": int(cand.size), "planted_found": hit,
                      "kept": int(G.sizes().s_kept)})
    cand_set = set(int(x) for x in cand)
    tp = len(truth & cand_set)
    rec = tp / len(truth) if truth else 0.0
    prec = tp / len(cand_set) if cand_set else 0.0
    f1 = 2 * prec * rec / (prec + rec) if prec + rec else 0.0
    line = {"workload": f"CTD-D stream of {args.steps} slices {st.dims2[0]}x{st.dims2[1]}, "
                        f"{st.nnz} nonzeros each, planted {len(st.planted_src)} x "
                        f"{len(truth)} block at steps {list(st.planted_steps)}; d = {args.d}, "
                        f"eps = {args.eps}",
            "recall": rec, "precision": prec, "f1": f1, "candidates": sorted(cand_set),
            "planted_dst": sorted(truth), "final_kept": int(G.sizes().s_kept),
            "step_nnz_per_s": tot_nnz / step_s,
            "detector_ms": {"median": 1e3 * float(np.median(det_s)), "max": 1e3 * max(det_s)},
            "phases_ms": ctd.profile_report()["phases"], "trace": trace}
    print(json.dumps(line), flush=True)


def sweep(args):
    """Sample-size sweep (Section 4, the experiment behind Fig. 4): CTD-S for
    s = 1 ... 1000 on a tensor shaped like the Haggle contact data of
    Table 3 (77 x 274 x 1567, 27,972 nonzeros; Zipf(1.2) ids, uniform time,
    Poisson(3)+1 counts) and on the 10^7-nonzero traffic tensor. Per s: the
    relative error, the kept count s~ (bounded by the rank of X_(1), at most
    77 on the first tensor), the device time of a call, and the memory of
    the result: the paper's memory usage (Eq. memoryEff) and the bytes of
    R as CSC, U dense, C as CSC with 16-bit rows."""
    tensors = [("haggle-shaped 77x274x1567, 27972 nnz",
                synth.traffic((77, 274, 1567), 27972, 1.2, 1.2, "poisson1", 2001, 3.0)),
               ("traffic 10000x10000x1000, 1e7 nnz", synth.traffic_10m())]
    if args.small_only:
        tensors = tensors[:1]
    svals = [1, 2, 5, 10, 20, 50, 100, 200, 500, 1000]
    out = []
    for name, coo in tensors:
        X = ctd.Coo.from_synth(coo)
        for _ in range(2):
            ctd.ctd_static(X, 1, 50, 1e-6, 0, ctd.CTD_FP32_BULK).free()
        rows = []
        for s_ in svals:
            times = []
            for rep in range(args.reps):
                _sync()
                t0 = time.perf_counter()
                F = ctd.ctd_static(X, 1, s_, 1e-6, rep, ctd.CTD_FP32_BULK)
                e = F.error()
                _sync()
                times.append(time.perf_counter() - t0)
                sz = F.sizes()
                if rep == 0:
                    row = {"s": s_, "s_unique": int(sz.s_unique), "s_kept": int(sz.s_kept),
                           "rel_error": e, "nnz_R": int(sz.nnz_R), "nnz_C": int(sz.nnz_C),
                           "memory_usage": memory_usage(F),
                           "memory_bytes": int(12 * sz.nnz_R + 8 * (sz.s_kept + 1)
                                               + 8 * sz.s_kept ** 2 + 6 * sz.nnz_C
                                               + 12 * (sz.n_cols + 1))}
                F.free()
            row["ms_median"] = 1e3 * float(np.median(times))
            rows.append(row)
        out.append({"tensor": name, "nnz": int(coo.nnz), "rows": rows})
    print(json.dumps({"workload": "CTD-S sample-size sweep, FP32_BULK, eps = 1e-6", "runs": out}),
          flush=True)


def protocol(args):
    """The paper's CTD-D vs CTD-S comparison (Section 4, performance of
    CTD-D): the first 80% of the time mode is the history, decomposed by
    CTD-S with s draws and used to seed CTD-D; the later slices arrive one
    at a time.  At each arriving slice: one CTD-D step with d = 0.01 s, and
    CTD-S recomputed on the whole tensor so far with s; device-resident
    inputs, both timed to the end of the call (error included).  Averages
    over the measured steps."""
    tensors = [("haggle-shaped 77x274x1567, 27972 nnz",
                synth.traffic((77, 274, 1567), 27972, 1.2, 1.2, "poisson1", 2001, 3.0), None),
               ("traffic 10000x10000x1000, 1e7 nnz", synth.traffic_10m(), args.big_steps)]
    import torch
    out = []
    for name, coo, max_steps in tensors:
        I, J, K = coo.dims
        kh = int(0.8 * K)
        s_ = args.s
        d = max(1, int(round(0.01 * s_)))
        hist = coo.subset(coo.k < kh)
        hist = synth.Coo3((I, J, kh), hist.i, hist.j, hist.k, hist.val)
        S = ctd.ctd_static(ctd.Coo.from_synth(hist), 1, s_, 1e-6, 0, ctd.CTD_FP32_BULK)
        S.error()
        G = ctd.Dynamic.from_static(S)
        # device copies of the whole tensor, in time order, for the CTD-S arm
        order = np.argsort(coo.k, kind="stable")
        dev = [torch.from_numpy(np.ascontiguousarray(a[order], dtype=np.int32)).cuda()
               for a in (coo.i, coo.j, coo.k, coo.val)]
        kcount = np.bincount(coo.k, minlength=K)
        upto = np.cumsum(kcount)
        steps = K - kh if max_steps is None else min(K - kh, max_steps)
        # warm both arms
        for _ in range(2):
            ctd.ctd_static(ctd.Coo((I, J, kh + 1), *(a[:upto[kh]] for a in dev)), 1, s_, 1e-6, 0,
                           ctd.CTD_FP32_BULK).free()
        td, ts, ed, es = [], [], [], []
        for t in range(kh, kh + steps):
            m = coo.k == t
            sl = synth.Coo3((I, J, 1), coo.i[m], coo.j[m], np.zeros(int(m.sum()), np.int64),
                            coo.val[m])
            X = ctd.Coo.from_synth(sl)
            _sync()
            t0 = time.perf_counter()
            G.step_slice(X, d, 1e-6)
            e1 = G.error()
            _sync()
            td.append(time.perf_counter() - t0)
            ed.append(e1)
            n = int(upto[t])
            Xs = ctd.Coo((I, J, t + 1), *(a[:n] for a in dev))
            _sync()
            t0 = time.perf_counter()
            F = ctd.ctd_static(Xs, 1, s_, 1e-6, 0, ctd.CTD_FP32_BULK)
            e2 = F.error()
            _sync()
            ts.append(time.perf_counter() - t0)
            es.append(e2)
            F.free()
        out.append({"tensor": name, "history_slices": kh, "steps_measured": steps, "s": s_,
                    "d": d, "ctd_d_ms": 1e3 * float(np.mean(td)),
                    "ctd_s_ms": 1e3 * float(np.mean(ts)),
                    "speedup": float(np.mean(ts) / np.mean(td)),
                    "ctd_d_error": float(np.mean(ed)), "ctd_s_error": float(np.mean(es)),
                    "ctd_d_kept_final": int(G.sizes().s_kept)})
    print(json.dumps({"workload": "CTD-D vs CTD-S, 80% history, d = 0.01 s, eps = 1e-6, FP32_BULK",
                      "runs": out}), flush=True)


# ---------------------------------------------------------------------------
# summaries of ncu output (text in, text out; no GPU)
# ---------------------------------------------------------------------------
def ncu_launch_summary(csv_path: str, top: int = 30) -> str:
    """Per kernel: launches, total time and share of an `ncu --metrics
    gpu__time_duration.sum --csv` launch list (serialized, cold-cache times:
    compare shares, not absolutes)."""
    import collections
    import csv
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, vi, ui = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Unit")
    mi = h.index("Metric Name") if "Metric Name" in h else None
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0,
             "msecond": 1.0, "s": 1e3, "second": 1e3}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= vi:
            continue
        if mi is not None and r[mi] != "gpu__time_duration.sum":
            continue  # other metrics of the same launch (a DRAM capture)
        name = r[ki].split("(")[0].replace("void ", "")
        agg[name][0] += 1
        agg[name][1] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
    tot = sum(v[1] for v in agg.values())
    lines = [f"{'kernel':48s} {'launches':>8s} {'total ms':>10s} {'share':>7s}"]
    for n, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1])[:top]:
        lines.append(f"{n:48s} {c:8d} {t:10.3f} {100 * t / tot:6.2f}%")
    lines.append(f"total: {sum(v[0] for v in agg.values())} launches, {tot:.3f} ms")
    return "\n".join(lines)


def ncu_dram_summary(csv_path: str, peak_gbs: float, top: int = 40) -> str:
    """Per kernel, from an `ncu --metrics dram__bytes_read.sum,
    dram__bytes_write.sum,gpu__time_duration.sum --csv` launch list: launches,
    mean duration, mean DRAM bytes moved and the rate they were moved at
    (serialized, cold-cache launches), and that rate as a fraction of
    `peak_gbs`."""
    import collections
    import csv
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ii, ki, mi = h.index("ID"), h.index("Kernel Name"), h.index("Metric Name")
    vi, ui = h.index("Metric Value"), h.index("Metric Unit")
    tscale = {"ns": 1e-9, "nsecond": 1e-9, "us": 1e-6, "usecond": 1e-6, "ms": 1e-3,
              "msecond": 1e-3, "s": 1.0, "second": 1.0}
    bscale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    launch = collections.defaultdict(lambda: [None, 0.0, 0.0])  # name, seconds, bytes
    for r in rows[hi + 1:]:
        if len(r) <= vi:
            continue
        rec = launch[r[ii]]
        rec[0] = r[ki].split("(")[0].replace("void ", "")
        v = float(r[vi].replace(",", ""))
        if r[mi] == "gpu__time_duration.sum":
            rec[1] += v * tscale.get(r[ui], 1e-9)
        elif r[mi].startswith("dram__bytes_"):
            rec[2] += v * bscale.get(r[ui], 1.0)
    agg = collections.defaultdict(lambda: [0, 0.0, 0.0])
    for name, sec, byt in launch.values():
        a = agg[name]
        a[0] += 1
        a[1] += sec
        a[2] += byt
    lines = [f"{'kernel':48s} {'launches':>8s} {'us/launch':>10s} {'MB/launch':>10s} "
             f"{'GB/s':>8s} {'of peak':>8s}"]
    for n, (c, sec, byt) in sorted(agg.items(), key=lambda x: -x[1][1])[:top]:
        rate = byt / sec / 1e9 if sec > 0 else 0.0
        lines.append(f"{n:48s} {c:8d} {1e6 * sec / c:10.1f} {byt / c / 1e6:10.2f} "
                     f"{rate:8.0f} {rate / peak_gbs:8.3f}")
    return "\n".join(lines)


def ncu_metrics_summary(rep_path: str, kernel_regex: str, names) -> dict:
    """Selected raw metrics of the captured launches of one kernel from an
    `ncu -o` report (read with `ncu -i ... --page raw --csv`)."""
    import csv
    import re
    import subprocess
    out = subprocess.run(["ncu", "-i", rep_path, "--page", "raw", "--csv"],
                         capture_output=True, text=True, check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    h = rows[0]
    res = []
    for r in rows[2:]:
        if not re.search(kernel_regex, r[h.index("Kernel Name")]):
            continue
        res.append({k: r[h.index(k)] for k in names if k in h})
    return {"launches": res}


def ncu_traffic_record(csv_path: str, kernels: str, scale: float, source: str) -> dict:
    """DRAM bytes (read + write) of the launches whose names match `kernels`
    in an `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --csv`
    log, summed over the captured launches and multiplied by `scale` (the
    ratio of the full workload's units to the captured case's), tagged with
    the hash of the kernels' source file."""
    import collections
    import csv
    import hashlib
    import re
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, mi, vi, ui = (h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"),
                      h.index("Metric Unit"))
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    per = collections.defaultdict(float)
    for r in rows[hi + 1:]:
        if len(r) <= vi or not re.search(kernels, r[ki]):
            continue
        if r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per[r[ki].split("(")[0].replace("void ", "")] += (
                float(r[vi].replace(",", "")) * unit.get(r[ui], 1.0))
    total = sum(per.values())
    sha = hashlib.sha256(open(source, "rb").read()).hexdigest()[:16]
    return {"source_sha": sha, "bytes_per_launch": total * scale, "captured_bytes": total,
            "scale": scale, "per_kernel_captured": dict(per)}


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    nt = sub.add_parser("ncu-traffic")
    nt.add_argument("csv")
    nt.add_argument("--kernels", required=True)
    nt.add_argument("--scale", type=float, required=True)
    nt.add_argument("--source", required=True)
    ns = sub.add_parser("ncu-summary")
    ns.add_argument("csv")
    ns.add_argument("--top", type=int, default=30)
    nd = sub.add_parser("ncu-dram")
    nd.add_argument("csv")
    nd.add_argument("--peak", type=float, required=True, help="GB/s (the measured copy)")
    nd.add_argument("--top", type=int, default=40)
    b = sub.add_parser("batched")
    b.add_argument("--count", type=int, default=256)
    b.add_argument("--workers", type=int, default=0)
    b.add_argument("--tune", action="store_true")
    sv = sub.add_parser("serving")
    sv.add_argument("--streams", type=int, default=64)
    sv.add_argument("--rate", type=float, default=2000.0)
    sv.add_argument("--seconds", type=float, default=2.0)
    sv.add_argument("--pool", type=int, default=96)
    sv.add_argument("--workers", type=int, default=8)
    sv.add_argument("--d", type=int, default=200)
    sm = sub.add_parser("stream")
    sm.add_argument("--steps", type=int, default=100)
    sm.add_argument("--scale", type=float, default=1.0)
    sm.add_argument("--d", type=int, default=400)
    sw = sub.add_parser("sweep")
    sw.add_argument("--reps", type=int, default=3)
    sw.add_argument("--small-only", action="store_true")
    pr = sub.add_parser("protocol")
    pr.add_argument("--s", type=int, default=500)
    pr.add_argument("--big-steps", type=int, default=40)
    dd = sub.add_parser("ddos")
    dd.add_argument("--steps", type=int, default=48)
    dd.add_argument("--scale", type=float, default=1.0)
    dd.add_argument("--d", type=int, default=10)
    dd.add_argument("--eps", type=float, default=0.15)
    args = ap.parse_args()
    if args.cmd == "ncu-summary":
        print(ncu_launch_summary(args.csv, args.top))
        return
    if args.cmd == "ncu-dram":
        print(ncu_dram_summary(args.csv, args.peak, args.top))
        return
    if args.cmd == "ncu-traffic":
        print(json.dumps(ncu_traffic_record(args.csv, args.kernels, args.scale, args.source)))
        return
    import torch
    torch.cuda.set_device(0)
    ctd.load()
    {"batched": batched, "serving": serving, "stream": stream, "ddos": ddos,
     "sweep": sweep, "protocol": protocol}[args.cmd](args)


if __name__ == "__main__":
    main()
