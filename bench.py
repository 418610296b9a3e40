#!/usr/bin/env python
"""Benchmark: k-th order statistics of one 2^27 float32 array on GB300.

Workload (the library's headline case): n = 2^27 float32, an equal-weight mixture of
N(0,1), lognormal(0,2) and Student-t(1) with 5% exact duplicates of one value and 10
+-inf entries (seed 4); one step selects the five ranks k in {1, n/100, [(n+1)/2],
99n/100, n}.  Inputs are resident in HBM when the timed region starts and are larger
than L2 (512 MiB vs 129 MB), so no flush is needed between steps.

value       whole-job Gelem/s = (selections x n) / time, device-timed with CUDA events
e2e         the same through the public API with the array in pinned HOST memory:
            host-to-device copy + selections + device-to-host read of the results every
            step (two device buffers: step s + 1's copy overlaps step s's selections)
roofline    the persistent select kernel: algorithmic bytes (passes x n x 4 + the finish's
            bytes: the compacted bracket written once and read once) /
            its CUDA-event duration, against the measured HBM copy bandwidth
cpu_baseline  the CPU oracle (numpy introselect on totalOrder keys) on three steps of
            the same workload, one selection a task on every host core

``--impl reference`` times that oracle as the reference arm.  Under torchrun (N > 1)
every rank runs an independent replica of the workload (the single-array path has no
data to exchange on one GPU per rank); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LOG2 = 27
FAMILY = "mixture"
SEED = 4


def ranks_for(n):
    return [1, n // 100, (n + 1) // 2, (99 * n) // 100, n]


def measured_peaks():
    for p in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        if os.path.exists(p):
            with open(p) as f:
                d = json.load(f)
            return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs; only
    samples whose timestamp falls inside the region (host clock) are summarised."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=20):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            deadline = time.time() + 5.0
            while not self.lines and time.time() < deadline:   # sampler running before the region
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        time.sleep(2.5 * self.period_ms / 1000.0)   # let the sample that covers the end arrive

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self):
        sm, mx, reasons, inside = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for recv, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            ts = self._stamp(parts[0])
            t = ts if ts is not None else recv
            if self.t0 is not None and not (self.t0 - 0.001 <= t <= (self.t1 or t) + 0.001):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            inside += 1
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": inside,
                "region_s": (self.t1 - self.t0) if self.t0 and self.t1 else None}


SELECT_SOURCES = ("select.cu", "select.cuh", "common.cuh", "elem.cuh", "layout.cuh", "bracket.cuh")


def select_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in SELECT_SOURCES:
        with open(os.path.join(ROOT, "paper_1104_2732_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def select_traffic():
    """Mean DRAM bytes (read + write) per launch of the select kernel over the five ranks of
    this workload, from the ncu capture summarised in profiles/select_kernel_f32_n2e27.md,
    when that capture was taken of the current kernel sources (their sha256 is recorded
    there); None otherwise."""
    import re
    path = os.path.join(ROOT, "profiles", "select_kernel_f32_n2e27.md")
    if not os.path.exists(path):
        return None, "no capture"
    with open(path) as f:
        text = f.read()
    m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    m2 = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    if not (m1 and m2):
        return None, "no capture"
    if m2.group(1) != select_sources_sha256():
        return None, "kernel changed since the capture"
    return int(m1.group(1)), "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean over the 5 ranks"


def cpu_oracle_steps(x, ks, steps, warm_steps=0):
    """The CPU oracle as it stands (oracle.select.select_kth, numpy) on `steps` steps of
    the workload -- every rank of ks on the whole array x -- one selection a task on every
    host core (x shared with the workers)."""
    tasks = [int(k) for _ in range(steps) for k in ks]
    warm = [int(k) for _ in range(max(1, warm_steps)) for k in ks]
    with SharedArray(x) as sh:
        wall, cores = oracle_pool_time(_oracle_rank_task, tasks, init=_shm_worker_init, initargs=sh.initargs,
                                       warm=warm)
    return {"value": len(tasks) * x.size / wall / 1e9, "unit": "Gelem/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of the workload (the {len(ks)} ranks on the whole array), "
                      "one selection a task", "seconds": wall, "ms_per_step": 1e3 * wall / steps}


HEADLINE_METRIC = "k-th select Gelem/s (n=2^27 float32)"


def headline_config(n, ks, world):
    """The `config` of the headline line (both arms)."""
    return {"workload": f"single-array k-th select, n=2^27 float32 {FAMILY} "
                        "(+5% duplicates, 10 +-inf), 5 ranks per step",
            "n": n, "ranks": ks, "parallelism": f"replicas x{world}",
            "l2": "input larger than L2 (no flush needed)"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands on the host cores, on the headline
    workload itself -- each step selects the five ranks on the whole 2^27 array, one
    selection a task of a process pool over every host core (W steps untimed, then K
    timed; the steps overlap on the cores, so ms_per_step is the wall time / K)."""
    import synth
    n = 1 << N_LOG2
    ks = ranks_for(n)
    x = synth.heavy_mixture(FAMILY, n, seed=SEED)
    cpu = cpu_oracle_steps(x, ks, steps=args.steps, warm_steps=args.warmup)
    value = cpu["value"]
    line = {
        "impl": "reference", "metric": HEADLINE_METRIC, "value": value,
        "unit": "Gelem/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": cpu["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(n, ks, world),
        "cpu_baseline": {"value": value, "unit": "Gelem/s", "cores": cpu["cores"], "kind": "oracle",
                         "sample": f"{args.steps} steps of the workload itself: the 5 ranks on the whole "
                                   "2^27 array, one selection a task"},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_segmented(gbs, ctx, torch, np, args):
    """4096 float32 normal arrays, sizes log-uniform in [1e3, 1e6], medians: the batched
    call captured in a CUDA graph (autotuned launch variant) against a plain loop of
    single-array selects over the same segments."""
    import synth
    x_host, off = synth.segmented(4096, seed=5)
    S = off.size - 1
    total = int(off[-1])
    x = torch.from_numpy(x_host).cuda()
    ot = torch.from_numpy(off).cuda()
    out = torch.empty(S, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        chosen, tune_ms = ctx.autotune_segmented(x, ot, None, out, stream=stream)
        ctx.select_segmented(x, ot, None, out, stream=stream)
    stream.synchronize()
    passes = ctx.segmented_passes(S)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        ctx.select_segmented(x, ot, None, out, stream=stream)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, args.steps)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the plain form: one single-array select per segment
    outs = torch.empty(S, device="cuda")
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for s_ in range(S):
        n_s = int(off[s_ + 1] - off[s_])
        ctx.select_kth(x[int(off[s_]):int(off[s_ + 1])], (n_s + 1) // 2, out=outs[s_:s_ + 1])
    p1.record()
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    same = bool(torch.equal(out.view(torch.int32), outs.view(torch.int32)))
    sizes = np.diff(off)
    big = sizes > ctx.segmented_variant()["smem_cap"]
    # the same batch with learned starting brackets for the medians (shipped model)
    learned = None
    model = os.path.join(ROOT, "paper_1104_2732_gb300", "bracket_model.bin")
    if os.path.exists(model):
        ctx.load_bracket_model(model)
        ctx.set_config(use_learned=1)
        outl = torch.empty(S, device="cuda")
        with torch.cuda.stream(stream):
            ctx.select_segmented(x, ot, None, outl, stream=stream)
        stream.synchronize()
        lpasses = np.array(ctx.segmented_passes(S))
        gl = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gl, stream=stream):
            ctx.select_segmented(x, ot, None, outl, stream=stream)
        for _ in range(3):
            gl.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            gl.replay()
        e1.record()
        torch.cuda.synchronize()
        lms_ = e0.elapsed_time(e1) / reps
        ctx.set_config(use_learned=0)
        learned = {"ms_per_batch": lms_, "value": S / (lms_ * 1e-3), "gelem_s": total / (lms_ * 1e-3) / 1e9,
                   "mean_passes_large_segments": float(lpasses[big].mean()) if big.any() else None,
                   "identical_to_plain_start": bool(torch.equal(out.view(torch.int32), outl.view(torch.int32))),
                   "speedup_vs_plain_start": ms / lms_}
    # CPU oracle (as it stands) on the whole batch, one segment a task on every host core
    cpu = None
    if not args.no_cpu:
        tasks = [(int(off[i]), int(off[i + 1])) for i in range(S)]
        with SharedArray(x_host) as sh:
            cpu_s, cores = oracle_pool_time(_oracle_segment_task, tasks, init=_shm_worker_init,
                                            initargs=sh.initargs, warm=tasks[:64])
        cpu = {"value": S / cpu_s, "unit": "selections/s", "gelem_s": total / cpu_s / 1e9, "cores": cores,
               "kind": "oracle", "sample": f"the whole batch: medians of all {S} segments, one a task"}
    return {
        "workload": f"{S} float32 normal arrays, sizes log-uniform [1e3, 1e6], total {total} elements, medians",
        "metric": "selections/s", "value": S / (ms * 1e-3), "gelem_s": total / (ms * 1e-3) / 1e9,
        "ms_per_batch": ms, "graph": True, "variant": chosen, "variant_ms": tune_ms,
        "plain_loop_ms": plain_ms, "plain_selections_s": S / (plain_ms * 1e-3),
        "speedup_vs_plain": plain_ms / ms, "identical_to_plain": same,
        "mean_passes_large_segments": float(np.mean(np.array(passes)[big])) if big.any() else None,
        "bytes_read_per_batch": int(sum(p * n * 4 for p, n in zip(passes, sizes))),
        "achieved_gbs": sum(p * n * 4 for p, n in zip(passes, sizes)) / (ms * 1e-3) / 1e9,
        "cpu_baseline": cpu,
        "learned_start": learned,
    }


def bench_lms(gbs, ctx, torch, np, args):
    """LMS / LTS of 2048 elemental candidates on n = 1e6, p = 8 (30% contaminated rows), in
    three forms: fused (TF32 x 3 tensor-core residuals recomputed in every cutting-plane
    pass, never written; brackets proposed from 8192 sampled rows, and for reference the
    start from the extremes), materialised (TF32 x 3 residual matrix + batched trimmed-sum
    select) and plain (float32 CUDA-core residuals + one single-array select per
    candidate and rank).  The chosen form is the faster of the first two; relative errors
    of sampled candidates against the float64 oracle for every form."""
    import synth
    from oracle import regression as oreg
    n, p, C = 1_000_000, 8, 2048
    X, y, beta = synth.regression(n, p, 6)
    th = np.ascontiguousarray(synth.elemental_thetas(X, y, C, 7).T)
    k, h = (n + 1) // 2, (n + p + 1) // 2
    Xt, yt, tt = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (X, y, th))

    def timed(fn, reps):
        fn()   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    reps = max(3, min(20, args.steps // 5))
    fused_ms, (lms_f, lts_f, fused_passes) = timed(lambda: ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h), reps)
    # the dominant kernel of the fused form: its compaction pass, timed by the library's
    # CUDA events on the call's stream (mean over a few calls)
    wms = []
    for _ in range(5):
        ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h)
        wms.append(ctx.lms_last_stats()["write_ms"])
    write_ms = statistics.mean(wms)
    clk_mhz = measured_peaks()[0].get("sm_max_mhz", 2070.0)
    lane_peak = 152 * 128 * float(clk_mhz) * 1e6
    ops = 9 * n * C
    roofline = {"bound": "alu", "kernel": "fused_pass_kernel<1, compaction>", "algorithmic_ops_per_launch": ops,
                "ops_per_candidate_row": 9, "achieved": ops / (write_ms * 1e-3), "peak": lane_peak,
                "unit": "lane-ops/s", "frac": ops / (write_ms * 1e-3) / lane_peak, "pass_ms": write_ms,
                "peak_derivation": "152 SMs x 128 FP32/INT32 lanes x the maximum SM clock",
                "ops": "residual subtract, square, s <= a, s > b, a < s <= b, sum and count below, "
                       "count above, count kept (the product runs on the tensor cores)"}
    # the same fused form started from the extremes (Algorithm 1, step 0) instead of the
    # sampled brackets
    ctx.set_config(lms_start=1)
    fx_ms, (lms_x, _, fx_passes) = timed(lambda: ctx.lms_lts_fused(Xt, yt, tt, k=k, h=h), reps)
    ctx.set_config(lms_start=0)
    fx_same = bool(torch.equal(lms_x.view(torch.int32), lms_f.view(torch.int32)))
    mat_ms, (lms_m, lts_m) = timed(lambda: ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=1, batched=True), reps)
    plain_ms, (lms_p, lts_p) = timed(lambda: ctx.lms_lts(Xt, yt, tt, k=k, h=h, precision=0, batched=False), 1)
    # the estimator search: LMS argmin and LTS refined by C-steps from the 10 best candidates
    search_ms, srch = timed(lambda: ctx.lms_lts_search(Xt, yt, tt, k=k, h=h, n_refine=10, max_steps=20),
                            max(2, reps // 4))
    srch = {kk: v.cpu().numpy() for kk, v in srch.items()}
    # the residual kernel alone (materialised form): bytes written against HBM
    S = torch.empty(C, n, dtype=torch.float32, device="cuda")
    res_ms, _ = timed(lambda: ctx.residual_sq(Xt, yt, tt, precision=1, out=S), reps)
    del S
    torch.cuda.empty_cache()
    peaks, kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    forms = {"fused": (lms_f, lts_f), "materialised": (lms_m, lts_m), "plain": (lms_p, lts_p)}
    forms = {kk: (a.cpu().numpy(), b.cpu().numpy()) for kk, (a, b) in forms.items()}
    rng = np.random.default_rng(8)
    n_sample = 8 if args.no_cpu else 64
    sample = rng.choice(C, n_sample, replace=False)
    err = {kk: [0.0, 0.0] for kk in forms}
    if args.no_cpu:
        t0 = time.perf_counter()
        oracle_vals = [_lms_oracle_candidate_on(X, y, th, c, k, h) for c in sample]
        cpu_s, cores = time.perf_counter() - t0, 1
    else:
        # the float64 oracle on every host core, one candidate a task
        cpu_s, cores = oracle_pool_time(_lms_oracle_task, [int(c) for c in sample], init=_lms_worker_init,
                                        initargs=(n, p, C, k, h))
        oracle_vals = [_lms_oracle_candidate_on(X, y, th, c, k, h) for c in sample[:8]]
        sample = sample[:8]
    for c, (wl, wt) in zip(sample, oracle_vals):
        for name, (l, t) in forms.items():
            err[name][0] = max(err[name][0], abs(l[c] / wl[0] - 1))
            err[name][1] = max(err[name][1], abs(t[c] / wt[0] - 1))
    chosen = "fused" if fused_ms <= mat_ms else "materialised"
    chosen_ms = min(fused_ms, mat_ms)
    return {
        "workload": "LMS/LTS, n=1e6, p=8, 30% contaminated rows, 2048 elemental candidates, k=(n+1)/2, h=(n+p+1)/2",
        "metric": "candidates/s", "value": C / (chosen_ms * 1e-3), "ms": chosen_ms, "chosen_form": chosen,
        "fused_ms": fused_ms, "fused_passes": fused_passes, "roofline": roofline,
        "fused_extremes_start": {"ms": fx_ms, "passes": fx_passes, "lms_identical": fx_same},
        "materialised_ms": mat_ms,
        "plain_value": C / (plain_ms * 1e-3), "plain_ms": plain_ms, "speedup_vs_plain": plain_ms / chosen_ms,
        "max_rel_err_vs_float64": {**{f"lms_{kk}": v[0] for kk, v in err.items()},
                                   **{f"lts_{kk}": v[1] for kk, v in err.items()},
                                   "candidates_sampled": int(sample.size), "target": 1e-5},
        "residual_kernel": {"ms": res_ms, "bytes_written": C * n * 4,
                            "gbs": C * n * 4 / (res_ms * 1e-3) / 1e9,
                            "hbm_frac": C * n * 4 / (res_ms * 1e-3) / 1e9 / hbm, "peak_kind": f"{kind} hbm_gbs"},
        "cpu_baseline": {"value": n_sample / cpu_s, "unit": "candidates/s", "cores": cores, "kind": "oracle",
                         "sample": f"float64 LMS and LTS of {n_sample} of the {C} candidates, one a task"},
        "search": {"ms": search_ms, "n_refine": 10, "max_steps": 20,
                   "lms_value": float(srch["lms_value"][0]), "lts_value": float(srch["lts_value"][0]),
                   "lts_start_index": int(srch["lts_index"][0]),
                   "lts_theta_max_abs_err_vs_beta": float(np.max(np.abs(srch["lts_theta"] - beta))),
                   "lms_theta_max_abs_err_vs_beta": float(np.max(np.abs(srch["lms_theta"] - beta)))},
        "fused_vs_materialised_max_rel_diff": {
            "lms": float(np.max(np.abs(forms["fused"][0] / forms["materialised"][0] - 1))),
            "lts": float(np.max(np.abs(forms["fused"][1] / forms["materialised"][1] - 1)))},
    }


_LMS = None


def _lms_oracle_candidate_on(X, y, th, c, k, h):
    """The float64 oracle's (LMS, LTS) objectives of candidate c."""
    from oracle import regression as oreg
    return oreg.lms_lts(X, y, th[c:c + 1].T, k, h)


def _lms_worker_init(n, p, C, k, h):
    """Pool worker start-up: the regression problem and its candidates, regenerated."""
    global _LMS
    import numpy as np
    import synth
    X, y, _ = synth.regression(n, p, 6)
    th = np.ascontiguousarray(synth.elemental_thetas(X, y, C, 7).T)
    _LMS = (X, y, th, k, h)


def _lms_oracle_task(c):
    X, y, th, k, h = _LMS
    return _lms_oracle_candidate_on(X, y, th, c, k, h)


KNN_N, KNN_P, KNN_M, KNN_K, KNN_C, KNN_SEED = 1 << 20, 8, 4096, 256, 16, 350


_KNN_DATA = None


def _knn_worker_init():
    """Pool worker start-up: the kNN problem, generated once per process."""
    global _KNN_DATA
    import synth
    _KNN_DATA = synth.knn_problem(KNN_N, KNN_P, KNN_M, KNN_C, seed=KNN_SEED)


def _knn_oracle_queries(idx):
    """CPU oracle for a few kNN queries (one task of the pool): float32 distances in the
    stated order, then the regression and the class vote of each query."""
    import numpy as np
    from oracle import knn as oknn
    X, Q, f, labels = _KNN_DATA
    D2 = oknn.squared_distances_f32(X, Q[idx]).astype(np.float64)
    oknn.regress_d2(D2, f, KNN_K, "inverse", 1e-6)
    oknn.classify_d2(D2, labels, KNN_K, KNN_C)
    return len(idx)


def oracle_pool_time(fn, tasks, init=None, initargs=(), warm=None):
    """Wall time of fn over tasks on every host core (a spawn-started process pool, so no
    process forks after CUDA is initialised; `init` runs in each worker before the timed
    region, and `warm` -- by default one task a worker -- runs there untimed) and the
    cores used."""
    import multiprocessing as mp
    cores = min(len(tasks), os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores, initializer=init, initargs=initargs) as pool:
        pool.map(fn, tasks[:cores] if warm is None else warm, chunksize=1)   # start-up, untimed
        t0 = time.perf_counter()
        pool.map(fn, tasks, chunksize=1)
        wall = time.perf_counter() - t0
    return wall, cores


_SHM = None


def _shm_worker_init(name, shape, dtype):
    """Pool worker start-up: attach the shared array (created by the parent, which alone
    unlinks it)."""
    global _SHM
    import numpy as np
    from multiprocessing import shared_memory
    h = shared_memory.SharedMemory(name=name)
    _SHM = (h, np.ndarray(shape, dtype=np.dtype(dtype), buffer=h.buf))


def _oracle_rank_task(k):
    """One oracle selection of rank k on the shared array (one task of the pool)."""
    from oracle import select as osel
    osel.select_kth(_SHM[1], k)
    return int(_SHM[1].size)


def _oracle_segment_task(bounds):
    """The oracle's median of one segment [s, e) of the shared array."""
    from oracle import select as osel
    s, e = bounds
    osel.select_kth(_SHM[1][s:e], (e - s + 1) // 2)
    return e - s


class SharedArray:
    """A host array in shared memory for the spawn pool's workers (context manager)."""

    def __init__(self, x):
        import numpy as np
        from multiprocessing import shared_memory
        self.h = shared_memory.SharedMemory(create=True, size=max(1, x.nbytes))
        self.a = np.ndarray(x.shape, dtype=x.dtype, buffer=self.h.buf)
        self.a[...] = x
        self.initargs = (self.h.name, x.shape, x.dtype.str)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        del self.a
        self.h.close()
        self.h.unlink()


def bench_knn(gbs, ctx, torch, np, args):
    """kNN regression (inverse-distance weights) and classification through d_(k) (Sec. 5):
    n = 2^20 points in p = 8 dimensions from 16 Gaussian clusters, 4096 queries, k = 256;
    the sampled-bracket form (one fused pass) against the plain form (distance rows written
    out, d_(k) by the segmented select, then the reduction pass).  Roofline of the fused
    pass kernel: 3p floating-point operations per (query, point) pair -- the distance in
    its stated order (p differences, p products, p - 1 sums) and one comparison -- against
    the float32 issue rate of the SMs (128 lanes each per clock at the sampled clock)."""
    import synth
    X, Q, f, labels = synth.knn_problem(KNN_N, KNN_P, KNN_M, KNN_C, seed=KNN_SEED)
    Xt, Qt, ft, lt = (torch.from_numpy(a).cuda() for a in (X, Q, f, labels))
    m = KNN_M

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    reps = max(3, min(20, args.steps // 5))
    res = {}
    pass_ms = []
    for start in (0, 1):
        ctx.set_config(knn_start=start)
        r_ms, (pred, kth) = timed(lambda: ctx.knn_regress(Xt, ft, Qt, KNN_K, weight="inverse"), reps)
        rec = ctx.knn_last_stats()
        if start == 0 and rec["pass_launches"]:
            pass_ms.append(rec["pass_ms"] / rec["pass_launches"])
        c_ms, (cls, votes, kth2) = timed(lambda: ctx.knn_classify(Xt, lt, KNN_C, Qt, KNN_K), reps)
        rec2 = ctx.knn_last_stats()
        if start == 0 and rec2["pass_launches"]:
            pass_ms.append(rec2["pass_ms"] / rec2["pass_launches"])
        res[start] = (r_ms, c_ms, pred.cpu().numpy(), cls.cpu().numpy(), kth.cpu().numpy(), rec)
    ctx.set_config(knn_start=0)
    same = bool(np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][4].view(np.uint32),
                                                                         res[1][4].view(np.uint32)))
    pred_diff = float(np.max(np.abs(res[0][2] - res[1][2]) / np.maximum(np.abs(res[1][2]), 1e-300)))
    # roofline of the fused pass kernel (ALU issue)
    clk = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10).stdout
        clk = float(out.strip().splitlines()[0])
    except Exception:
        clk = 2070.0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sms * 128 * clk * 1e6
    ops = 3 * KNN_P * KNN_M * KNN_N
    pms = statistics.median(pass_ms) if pass_ms else None
    achieved = ops / (pms * 1e-3) if pms else None
    # CPU oracle: 64 queries on every host core
    cpu = None
    if not args.no_cpu:
        tasks = [[i] for i in range(0, 64 * 16, 16)]
        wall, cores = oracle_pool_time(_knn_oracle_queries, tasks, init=_knn_worker_init)
        cpu = {"value": len(tasks) / wall, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(tasks)} of the {KNN_M} queries (regression and vote each), one query per task"}
    return {
        "workload": f"kNN, n=2^20 points, p={KNN_P}, {KNN_C} Gaussian clusters, {KNN_M} queries, k={KNN_K}; "
                    "regression with inverse-distance weights and class vote",
        "metric": "queries/s", "value": m / (res[0][0] * 1e-3), "regress_ms": res[0][0], "classify_ms": res[0][1],
        "classify_queries_s": m / (res[0][1] * 1e-3), "passes": res[0][5]["passes"],
        "plain_queries": res[0][5]["plain_queries"],
        "plain_form": {"regress_ms": res[1][0], "classify_ms": res[1][1], "value": m / (res[1][0] * 1e-3),
                       "passes": res[1][5]["passes"]},
        "speedup_vs_plain": res[1][0] / res[0][0], "identical_classes_and_kth": same,
        "max_rel_pred_diff_vs_plain": pred_diff,
        "roofline": {"bound": "alu", "kernel": "knn_pass_kernel<8,4>", "achieved": achieved, "peak": peak_ops,
                     "unit": "FP32 lane-ops/s", "frac": achieved / peak_ops if achieved else None,
                     "algorithmic_ops_per_launch": ops, "pass_ms": pms,
                     "peak_derivation": f"{sms} SMs x 128 FP32 lanes x {clk:.0f} MHz (max SM clock)"},
        "cpu_baseline": cpu,
    }


def bench_learned(gbs, ctx, torch, np, args, x_big=None):
    """Median select from the data's extremes against the same select started from the
    trained network's proposed bracket (results must be identical), on (1) held-out
    arrays of the training distribution (generator seeds 2e6 + i, n in [2^20, 2^24]) with
    L2 flushed before every timed select, and (2) the 2^27 single-array workload."""
    from paper_1104_2732_gb300 import train_bracket as tb
    model = os.path.join(ROOT, "paper_1104_2732_gb300", "bracket_model.bin")
    if not os.path.exists(model):
        return {"unavailable": "no trained model"}
    ctx.load_bracket_model(model)
    flush = torch.empty(1 << 26, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    count = 1000
    rng = np.random.default_rng(2 * 10 ** 6)
    buf = torch.empty(1 << 24, device="cuda")
    outs = torch.empty(2, device="cuda")
    passes = {0: [], 1: []}
    ms = {0: 0.0, 1: 0.0}
    elems = 0
    same = True
    used = 0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(count):
        n, fam, p0, p1, p2, loc, scale = tb.draw_params(rng)
        x = buf[:n]
        ctx.generate_training_array(x, fam, p0, p1, p2, loc, scale, seed=2 * 10 ** 6 + i)
        k = (n + 1) // 2
        elems += n
        for mode in (0, 1):
            ctx.set_config(use_learned=mode)
            flush.zero_()
            ev[0].record()
            ctx.select_kth(x, k, out=outs[mode:mode + 1])
            ev[1].record()
            st = ctx.last_stats()      # synchronises
            ms[mode] += ev[0].elapsed_time(ev[1])
            passes[mode].append(st["passes"])
            used += int(mode == 1 and st["learned"] == 1)
        same = same and bool(outs[0].view(torch.int32) == outs[1].view(torch.int32))
    row = {
        "workload": f"{count} held-out arrays, n log-uniform [2^20, 2^24], normal / Student-t / lognormal / "
                    "contaminated, random location and scale; medians; L2 flushed before each select",
        "metric": "selections/s", "value": count / (ms[1] * 1e-3), "plain_value": count / (ms[0] * 1e-3),
        "speedup_vs_plain": ms[0] / ms[1],
        "mean_passes_learned": float(np.mean(passes[1])), "mean_passes_plain": float(np.mean(passes[0])),
        "p90_passes_learned": float(np.percentile(passes[1], 90)),
        "p90_passes_plain": float(np.percentile(passes[0], 90)),
        "proposal_valid_fraction": used / count, "identical_results": same,
        "gelem_s_learned": elems / (ms[1] * 1e-3) / 1e9, "gelem_s_plain": elems / (ms[0] * 1e-3) / 1e9,
    }
    if x_big is not None:
        n = x_big.numel()
        k = (n + 1) // 2
        res = {}
        for mode in (0, 1):
            ctx.set_config(use_learned=mode)
            for _ in range(2):
                ctx.select_kth(x_big, k, out=outs[mode:mode + 1])
            torch.cuda.synchronize()
            ev[0].record()
            for _ in range(5):
                ctx.select_kth(x_big, k, out=outs[mode:mode + 1])
            ev[1].record()
            st = ctx.last_stats()
            res[mode] = (ev[0].elapsed_time(ev[1]) / 5, st["passes"], st["learned"])
        row["median_2e27"] = {"ms_plain": res[0][0], "ms_learned": res[1][0], "passes_plain": res[0][1],
                              "passes_learned": res[1][1], "proposal": res[1][2],
                              "speedup": res[0][0] / res[1][0],
                              "identical": bool(outs[0].view(torch.int32) == outs[1].view(torch.int32))}
    ctx.set_config(use_learned=0)
    return row


def _bits(t, torch):
    return t.view(torch.int32 if t.dtype == torch.float32 else torch.int64)


def bench_small(gbs, ctx, torch, np, args):
    """n = 10^6 uniform [0, 1) float32 (seed 0), median (k = 500000): 4 MB, L2-resident and
    latency-bound.  Device time per selection over 200 back-to-back calls, passes, and the
    CPU oracle on the same array (best / median of 10 runs after 2 warm-ups)."""
    import synth
    from oracle import select as osel
    x_h = synth.uniform(1_000_000, seed=0)
    x = torch.from_numpy(x_h).cuda()
    k = 500_000
    out = torch.empty(1, device="cuda")
    for _ in range(5):
        ctx.select_kth(x, k, out=out)
    st = ctx.last_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record()
    for _ in range(reps):
        ctx.select_kth(x, k, out=out)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    for _ in range(2):
        osel.select_kth(x_h, k)
    cpu = []
    for _ in range(10):
        t0 = time.perf_counter()
        want = osel.select_kth(x_h, k)
        cpu.append((time.perf_counter() - t0) * 1e6)
    same = bool(np.asarray(out.cpu().numpy()[0], np.float32).view(np.uint32)
                == np.asarray(want, np.float32).view(np.uint32))
    return {"workload": "median of n=1e6 uniform [0,1) float32, seed 0", "metric": "us/selection",
            "value": us, "passes": st["passes"], "how": st["how"], "grid": st["grid"],
            "cpu_oracle_us_best": min(cpu), "cpu_oracle_us_median": statistics.median(cpu), "cpu_cores": 1,
            "identical_to_oracle": same}


def bench_f64(gbs, ctx, torch, np, args):
    """n = 2^26 float64 mixture (seed 4), the five ranks per step, 10 steps; bytes per
    call = (passes x n + compacted) x 8 against the measured HBM bandwidth; torch.sort of
    the same array as the comparator."""
    import synth
    n = 1 << 26
    x = torch.from_numpy(synth.heavy_mixture(FAMILY, n, seed=SEED, dtype=np.float64)).cuda()
    ctx.reserve(n, 8)
    ks = ranks_for(n)
    out = torch.empty(len(ks), dtype=torch.float64, device="cuda")
    recs = []
    for i, k in enumerate(ks):
        ctx.select_kth(x, k, out=out[i:i + 1])
        recs.append(ctx.last_stats())
    steps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for i, k in enumerate(ks):
            ctx.select_kth(x, k, out=out[i:i + 1])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    alg = sum((r["passes"] * n + 2 * r["finish_pop"]) * 8 for r in recs)
    peaks, kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    for _ in range(2):
        torch.sort(x)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(3):
        torch.sort(x)
    s1.record()
    torch.cuda.synchronize()
    sort_ms = s0.elapsed_time(s1) / 3
    res = {"workload": f"n=2^26 float64 {FAMILY} (+5% duplicates, 10 +-inf), ranks {ks}", "metric": "Gelem/s",
           "value": len(ks) * n / (ms * 1e-3) / 1e9, "ms_per_step": ms, "passes": [r["passes"] for r in recs],
           "hbm_frac": alg / (ms * 1e-3) / 1e9 / hbm, "peak_kind": f"{kind} hbm_gbs",
           "torch_sort_ms": sort_ms, "speedup_vs_torch_sort_per_selection": sort_ms / (ms / len(ks))}
    del x
    torch.cuda.empty_cache()
    return res


def bench_families(gbs, ctx, torch, np, args):
    """The three single-family 2^27 float32 arrays (normal seed 1, lognormal(0,2) seed 2,
    Student-t nu=1 seed 3; each +5% duplicates of its median and 10 +-inf), five ranks
    per step, 5 steps each."""
    import synth
    n = 1 << N_LOG2
    ks = ranks_for(n)
    out = torch.empty(len(ks), dtype=torch.float32, device="cuda")
    res = {}
    for fam, seed in (("normal", 1), ("lognormal", 2), ("cauchy", 3)):
        x = torch.from_numpy(synth.heavy_mixture(fam, n, seed=seed)).cuda()
        recs = []
        for i, k in enumerate(ks):
            ctx.select_kth(x, k, out=out[i:i + 1])
            recs.append(ctx.last_stats())
        steps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            for i, k in enumerate(ks):
                ctx.select_kth(x, k, out=out[i:i + 1])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[fam] = {"gelem_s": len(ks) * n / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                    "passes": [r["passes"] for r in recs], "how": [r["how"] for r in recs]}
        del x
    torch.cuda.empty_cache()
    return {"workload": "2^27 float32 single-family arrays, 5 ranks per step", "metric": "Gelem/s", **res}


def bench_drivers(gbs, ctx, torch, np, args):
    """The paper's comparison of drivers (Sec. 4, Tables 1-2 and Discussion) on GB300: the
    median of 2^25 normal float32 elements, plain and with one element set to 1e9, 1e20 or
    3e38, selected by the host-driven state machine (one device pass per iterate, the
    totals read back between passes, as the paper's implementation did) with each driver:
    Kelley's cutting plane, bisection, Brent's root-finder, Kelley on u = log1p(x - x_(1)).
    Passes and host wall time per selection; results must all equal the oracle's."""
    from oracle import select as osel
    from paper_1104_2732_gb300.sharded import GpuBackend, select_kth_sharded
    import synth
    n = 1 << 25
    base = synth.paper_distribution("normal", n, 75)
    k = (n + 1) // 2
    out = {}
    for big in (None, 1e9, 1e20, 3e38):
        x = base.copy()
        if big is not None:
            x[n // 3] = np.float32(big)
        want = np.float32(osel.select_kth(x, k)).view(np.uint32)
        xt = torch.from_numpy(x).cuda()
        row = {}
        for driver in ("kelley", "bisect", "brent", "log"):
            select_kth_sharded([xt], k, GpuBackend(ctx), elem_bytes=4, driver=driver)   # warm-up
            torch.cuda.synchronize()
            trace = []
            t0 = time.perf_counter()
            r = select_kth_sharded([xt], k, GpuBackend(ctx), elem_bytes=4, driver=driver, trace=trace)
            ms = (time.perf_counter() - t0) * 1e3
            row[driver] = {"passes": len(trace) + 1, "ms": ms,
                           "identical_to_oracle": bool(np.float32(r).view(np.uint32) == want)}
        out["none" if big is None else f"{big:g}"] = row
        del xt
    return {"workload": "median of 2^25 normal float32, plain and with one outlier; host-driven passes",
            "metric": "passes per selection (the pass-0 statistics pass included)", "rows": out}


def bench_sharded(gbs, ctx, torch, np, args, x):
    """The 2^27 array as four shards on this device, median: the device-resident loop
    (per-shard passes into one device accumulator, the state advanced on the device, the
    phase read back every 4 passes) and the host-driven loop (totals summed on the host
    between passes); wall time of each, identical result to the single-array select
    required."""
    from paper_1104_2732_gb300.sharded import GpuBackend, select_kth_sharded
    n = x.numel()
    m = n // 4
    shards = [x[i * m:(i + 1) * m] if i < 3 else x[3 * m:] for i in range(4)]
    k = (n + 1) // 2
    single = float(ctx.select_kth(x, k).item())
    trace = []
    select_kth_sharded(shards, k, GpuBackend(ctx), elem_bytes=4)      # warm-up
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        trace = []
        got = select_kth_sharded(shards, k, GpuBackend(ctx), elem_bytes=4, trace=trace)
    ms = (time.perf_counter() - t0) / reps * 1e3
    # the device-resident loop on the same shards (no process group: one rank)
    from paper_1104_2732_gb300.sharded import select_kth_sharded_device
    info = {}
    select_kth_sharded_device(shards, k, ctx, elem_bytes=4, info=info)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        info = {}
        got_d = select_kth_sharded_device(shards, k, ctx, elem_bytes=4, info=info)
    ms_d = (time.perf_counter() - t0) / reps * 1e3
    same = lambda v: bool(np.float32(v).view(np.uint32) == np.float32(single).view(np.uint32))
    return {"workload": "median of the 2^27 float32 array split into 4 shards on one device",
            "metric": "ms/selection (host wall clock)", "value": ms_d, "form": "device-resident loop",
            "cutting_plane_passes": info["passes"], "launched_passes": info["launched_passes"],
            "identical_to_single_array": same(got_d),
            "host_loop": {"ms": ms, "cutting_plane_passes": len(trace), "identical_to_single_array": same(got)},
            "speedup_vs_host_loop": ms / ms_d}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--only-single", action="store_true", help="time the single-array select only")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1104_2732_gb300 as gbs
    import synth

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    n = 1 << N_LOG2
    ks = ranks_for(n)
    x_host = synth.heavy_mixture(FAMILY, n, seed=SEED + rank)
    x = torch.from_numpy(x_host).cuda()
    ctx = gbs.Context(local_rank)
    ctx.reserve(n, 4)
    out = torch.empty(len(ks), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        for i, k in enumerate(ks):
            ctx.select_kth(x, k, out=out[i:i + 1])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # per-call records (passes, per-pass timestamps) from one untimed step
    records = []
    for i, k in enumerate(ks):
        ctx.select_kth(x, k, out=out[i:i + 1])
        records.append(ctx.last_stats())

    # ---------------- device-timed region ----------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps * len(ks))]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        clk.start()
        start.record(stream)
        j = 0
        for _ in range(args.steps):
            for i, k in enumerate(ks):
                ev[j][0].record(stream)
                ctx.select_kth(x, k, out=out[i:i + 1])
                ev[j][1].record(stream)
                j += 1
        stop.record(stream)
        torch.cuda.synchronize()
        clk.stop()
    if world > 1:
        dist.barrier()
    ms = start.elapsed_time(stop)
    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    launch_ms = [a.elapsed_time(b) for a, b in ev]

    total_elems = world * args.steps * len(ks) * n
    value = total_elems / (ms_max * 1e-3) / 1e9

    # ---------------- roofline of the select kernel ----------------
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # passes x n x 4 + the finish's bytes (the compacted bracket written once and read once;
    # the radix rounds after the first two read only the second-level copy)
    bytes_per_call = [(r["passes"] * n + 2 * r["finish_pop"]) * 4 for r in records]
    alg_bytes = args.steps * sum(bytes_per_call)
    achieved = alg_bytes / (sum(launch_ms) * 1e-3) / 1e9
    traffic, traffic_src = select_traffic()
    # per-pass bandwidth from the kernel's own timestamps (pass 0 and Kelley passes)
    pass_gbs, stream_gbs, overhead_us = [], [], []
    for r in records:
        t = r["t_ns"]
        for i in range(min(r["passes"], len(t) - 1)):
            dt = (t[i + 1] - t[i]) * 1e-9
            if dt > 0:
                pass_gbs.append(n * 4 / dt / 1e9)
            # cutting-plane pass i-1 (pass 0 has no separate stamp): streaming part alone
            if i >= 1 and i - 1 < len(r["t_stream_ns"]) and r["t_stream_ns"][i - 1]:
                ds = (r["t_stream_ns"][i - 1] - t[i]) * 1e-9
                if ds > 0:
                    stream_gbs.append(n * 4 / ds / 1e9)
                    overhead_us.append(round((dt - ds) * 1e6, 1))

    # ---------------- end to end through the public API, host buffers ----------------
    # every step copies its array from pinned host memory, selects the five ranks and
    # reads the results back; two device buffers let the copy of step s + 1 (on its own
    # stream) run while step s selects
    pinned = torch.from_numpy(x_host).pin_memory()
    res_host = torch.empty((2, len(ks)), dtype=torch.float32).pin_memory()
    xb = [x, torch.empty_like(x)]
    outs = [out, torch.empty_like(out)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_steps = max(2, args.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    with torch.cuda.stream(copy_stream):
        xb[0].copy_(pinned, non_blocking=True)
    copied[0].record(copy_stream)
    for s_ in range(e2e_steps):
        b = s_ % 2
        if s_ + 1 < e2e_steps:
            nb = 1 - b
            if s_ >= 1:
                copy_stream.wait_event(freed[nb])   # step s - 1 is done with that buffer
            with torch.cuda.stream(copy_stream):
                xb[nb].copy_(pinned, non_blocking=True)
            copied[nb].record(copy_stream)
        stream.wait_event(copied[b])
        for i, k in enumerate(ks):
            ctx.select_kth(xb[b], k, out=outs[b][i:i + 1])
        freed[b].record(stream)
        res_host[b].copy_(outs[b], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_same = bool(torch.equal(res_host[(e2e_steps - 1) % 2].view(torch.int32), out.cpu().view(torch.int32)))
    e2e_value = world * len(ks) * n / (e2e_ms * 1e-3) / 1e9

    # ---------------- comparator: full on-device sort of the same array ----------------
    torch.cuda.synchronize()
    for _ in range(2):
        torch.sort(x)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(3):
        torch.sort(x)
    s1.record(stream)
    torch.cuda.synchronize()
    sort_ms = s0.elapsed_time(s1) / 3

    # ---------------- other rows of the hot path (one GPU: the replicas of N > 1 time only
    # the headline, so the N GPUs are not held for rows that say nothing about scaling) ----
    rows = {}
    if not args.only_single and world == 1:
        del pinned
        rows["small_n1e6"] = bench_small(gbs, ctx, torch, np, args)
        rows["sharded_4_shards"] = bench_sharded(gbs, ctx, torch, np, args, x)
        rows["drivers"] = bench_drivers(gbs, ctx, torch, np, args)
        rows["learned_bracket"] = bench_learned(gbs, ctx, torch, np, args, x_big=x)
        rows["segmented"] = bench_segmented(gbs, ctx, torch, np, args)
        rows["lms_lts"] = bench_lms(gbs, ctx, torch, np, args)
        rows["knn"] = bench_knn(gbs, ctx, torch, np, args)
        rows["f64_n2e26"] = bench_f64(gbs, ctx, torch, np, args)
        rows["families_f32"] = bench_families(gbs, ctx, torch, np, args)

    # ---------------- CPU oracle baseline (rank 0 only) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_steps(x_host, ks, steps=3)

    if rank == 0:
        sel_ms = [sum(launch_ms[i::len(ks)]) / args.steps for i in range(len(ks))]
        line = {
            "metric": HEADLINE_METRIC,
            "value": value,
            "unit": "Gelem/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(3, args.warmup),
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": headline_config(n, ks, world),
            "gpu_launches": args.steps * len(ks),
            "e2e": {"value": e2e_value, "unit": "Gelem/s", "h2d_bytes_per_step": n * 4,
                    "d2h_bytes_per_step": len(ks) * 4, "ms_per_step": e2e_ms,
                    "pipelined": "two device buffers: step s + 1's host-to-device copy overlaps step s",
                    "results_match_device_timed_run": e2e_same},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes_per_launch": alg_bytes / (args.steps * len(ks)),
                         "traffic_source": traffic_src,
                         "peak_kind": f"{peak_kind} hbm_gbs", "kernel": "select_kernel<float>"},
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "rows": rows,
            "detail": {
                "ms_per_selection": dict(zip([str(k) for k in ks], sel_ms)),
                "passes": [r["passes"] for r in records],
                "how": [r["how"] for r in records],
                "finish_pop": [r["finish_pop"] for r in records],
                "pass_gbs_median": statistics.median(pass_gbs) if pass_gbs else None,
                "pass_gbs": [round(v, 1) for v in pass_gbs],
                "stream_gbs": [round(v, 1) for v in stream_gbs],
                "pass_overhead_us": overhead_us,
                "torch_sort_ms": sort_ms,
                "torch_sort_gelems": n / (sort_ms * 1e-3) / 1e9,
                "median_select_ms": sel_ms[2],
                "speedup_vs_torch_sort_median": sort_ms / sel_ms[2],
            },
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
