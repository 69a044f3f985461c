"""Benchmark: batched exact hypothesis evaluation on one GB300 (or N, one process per GPU).

Workload (default): 1,000,000 individuals, 100 concepts, 16 roles with
Poisson(6) out-degree (+ inverses), 8 data properties uniform [0, 1000],
10,000 / 10,000 examples; every step evaluates and scores one batch of 4,096
seeded hypotheses of postfix length uniform 1..40 and depth uniform 1..8 with
shared sub-concepts at rate 0.3.  Inputs are synthetic (seeded generators),
and larger than L2 (the KB alone is ~0.95 GB), so no L2 flush is needed.

Prints ONE JSON line (rank 0):
  value          hypotheses/s, device-timed, KB and plans resident in HBM
                 (CUDA events on the launching stream around graph replays)
  e2e            the same metric through hedl_score_batch from HOST programs
                 (planning, plan upload, launch, D2H of the counts), wall clock
  roofline       achieved = algorithmic bytes of a launch (the plan's byte
                 model) / mean launch time, against the measured HBM peak
  cpu_baseline   the oracle on the host cores on a bounded sample
  plain          the one-launch-per-operation path on the same batches
``--impl reference`` times the oracle instead (the reference arm).
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
from dataclasses import replace as dc_replace

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("batched exact evaluation: N=1,000,000 individuals, 100 concepts, 16 roles Poisson(6) + inverses, "
            "8 props U[0,1000], 10k/10k examples; 4,096 hypotheses per step, length U[1,40], depth U[1,8], "
            "shared sub-concepts 0.3")
METRIC = "exact hypotheses/sec"
UNIT = "hyp/s"
BATCH = 4096


def shard_batches(rank: int, world: int, warmup: int, steps: int):
    """Batch indices this rank evaluates: warm-up ones, then timed ones; disjoint across ranks."""
    per = warmup + steps
    base = rank * per
    return list(range(base, base + warmup)), list(range(base + warmup, base + per))


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_bf16_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def mlp_forward_timing(s, X):
    """CUDA-event time of the surrogate's forward over X on each GEMM engine, with the
    tensor roofline of the dense layers (2 x B x (512*512*2 + 512*2) flops)."""
    import torch
    import paper_2412_00802_gb300 as H
    B = X.shape[0]
    Y = torch.empty((B, 2), dtype=torch.float32, device=X.device)
    ws = s._workspace(B)
    flops = 2.0 * B * (512 * 512 * 2 + 512 * 2)
    peak, kind = measured_bf16_tflops()
    out = {"rows": B, "flops": flops, "peak_tflops": peak, "peak_kind": f"{kind} bf16 (MEASURED_PEAKS.json bf16_tflops)"}
    stream = torch.cuda.current_stream(X.device)
    for name, eng, reps in (("tcgen05", H.HEDL_GEMM_TCGEN05, 60), ("mma_sync", H.HEDL_GEMM_MMA_SYNC, 10)):
        H.hedl_mlp_set_gemm(s.mlp, eng)
        for _ in range(5):
            H.hedl_mlp_forward(s.mlp, X, Y, ws)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        with ClockSampler(X.device.index or 0) as clk:
            t_end = time.perf_counter() + 1.0    # ~1 s of forwards first, so the clock samples see the load
            while time.perf_counter() < t_end:
                for _ in range(20):
                    H.hedl_mlp_forward(s.mlp, X, Y, ws)
                torch.cuda.synchronize()
            for a, b in ev:              # one forward per event pair; the median is reported
                a.record(stream)
                H.hedl_mlp_forward(s.mlp, X, Y, ws)
                b.record(stream)
            torch.cuda.synchronize()
        t = sorted(a.elapsed_time(b) for a, b in ev)
        ms = statistics.median(t)
        out[name] = {"ms": ms, "tflops": flops / ms / 1e9, "frac": flops / ms / 1e9 / peak, "forwards": reps,
                     "ms_min": t[0], "ms_max": t[-1], "clocks": clk.summary()}
    H.hedl_mlp_set_gemm(s.mlp, H.HEDL_GEMM_TCGEN05)
    H.hedl_mlp_status(s.mlp)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(workload_key: str, tuning: dict):
    """The committed ncu figures of the interpreter launch (profiles/traffic.json: DRAM bytes per
    launch, and the L2 throughput share if captured), if they were taken on the current
    interpreter sources with the same launch shape; else None (stale counters are not reused)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        from paper_2412_00802_gb300 import build
        with open(p) as f:
            d = json.load(f)
        e = d.get(workload_key)
        if e and e.get("interpreter_digest") == build.interpreter_digest() and e.get("tuning") == tuning:
            return e
    except Exception:
        pass
    return None


def _r(x, nd: int = 4):
    """A number rounded to nd significant digits (None stays None) for the compact summary."""
    if x is None or isinstance(x, bool):
        return x
    if isinstance(x, int):
        return x
    return float(f"{x:.{nd}g}")


def make_workload(seed_kb: int = 3):
    from synth import kb as K
    return K.generate(K.CONFIGS["batch"])


def make_batch(kb, idx: int, gen=None, count: int = None):
    from synth import hyps
    return hyps.batch_hyps(kb, 1003, idx, count or BATCH, gen=gen)


def cpu_baseline(kb, progs, budget_s: float = 12.0, single_budget_s: float = 4.0):
    """The oracle (as it stands) on all host cores over a bounded sample of the batch (the paper's
    multi-threaded CPU evaluator's analog), and on one thread (its single-threaded baseline's)."""
    import oracle
    from synth import programs as P
    okb = oracle.from_synth(kb)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def run(threads, chunk, budget):
        done, t0 = 0, time.perf_counter()
        while done < len(progs) and time.perf_counter() - t0 < budget:
            sub = progs[done:done + chunk]
            flat, offs = P.pack_batch(sub)
            oracle.eval_batch(okb, flat, offs, threads=threads)
            done += len(sub)
        return done, time.perf_counter() - t0

    done, dt = run(cores, max(cores, 16), budget_s)
    done1, dt1 = run(1, 1, single_budget_s)
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} hypotheses of a 4,096-hypothesis batch of this workload, "
                      f"hypothesis-parallel on {cores} host threads ({dt:.1f} s)",
            "single_thread": {"value": done1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {done1} hypotheses of the same batch on one thread ({dt1:.1f} s)"}}


def _pack(progs):
    from synth import programs as P
    return P.pack_batch(progs)


def surrogate_round(args, dev):
    """One surrogate-ranked round on a planted KB with the single-hypothesis workload's
    distributions: train on engine-scored hypotheses, rank 65,536 candidates, score the
    predicted top 5 % exactly; recall@100 against the exact ranking and best-found/sec
    against the plain batched path (every candidate scored, in generation order)."""
    import torch
    import paper_2412_00802_gb300 as H
    from paper_2412_00802_gb300 import surrogate as sg
    from oracle import surrogate as OS
    from synth import hyps, kb as K
    full = not args.surrogate_small
    cfg = K.CONFIGS["surrogate"] if full else K.CONFIGS["surrogate"].scaled(1_000_000)
    t0 = time.perf_counter()
    kb = K.generate(cfg)
    gen_s = time.perf_counter() - t0
    dkb = H.DeviceKB.from_synth(kb, device=str(dev))
    tg = hyps.TreeGen(kb, 404, share=0.3)
    n_train = args.surrogate_train or (1_000_000 if full else 65_536)
    B = 4096
    t0 = time.perf_counter()
    Xs, Ts = [], []
    s = sg.Surrogate(seed=4, device=str(dev), grid=sg.threshold_grid(kb.prop_vals))
    s.fit_statistics(dkb, kb.n_concepts)      # the KB's per-symbol exact scores (an encoder input)
    for b in range(n_train // B):
        flat, offs = _pack(hyps.batch_hyps(kb, 404, b, B, gen=tg))
        _, T = sg.exact_scores(dkb, flat, offs)
        Xs.append(s.encode(flat, offs))
        Ts.append(T)
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    torch.cuda.synchronize()
    score_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = s.train(X, T, epochs=40, batch=B, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    cand = hyps.batch_hyps(kb, 405, 0, 65_536, gen=tg)
    cflat, coffs = _pack(cand)
    # plain batched path: all candidates, in generation order
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_at, exact = [], []
    for b0 in range(0, len(cand), B):
        f, o = _pack(cand[b0:b0 + B])
        _, T = sg.exact_scores(dkb, f, o)
        exact.append(T.cpu().numpy())
        done_at.append(time.perf_counter() - t0)
    exact = np.concatenate(exact)
    order = OS.rank_order(exact[:, 0], exact[:, 1], cand)
    best = order[0]
    plain_s = done_at[best // B]
    # surrogate path: encode, predict, keep the top 5 %, score those exactly
    k = int(round(0.05 * len(cand)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Y = s.predict(s.encode(cflat, coffs))
    sel = s.select(Y, k).cpu().numpy()
    f, o = _pack([cand[i] for i in sel])
    _, Tsel = sg.exact_scores(dkb, f, o)
    Tsel = Tsel.cpu().numpy()
    sur_s = time.perf_counter() - t0
    found = bool(best in set(sel.tolist()))
    fwd = mlp_forward_timing(s, s.encode(cflat, coffs))
    top_pred = np.argsort(-Y[:, 0].cpu().numpy(), kind="stable")[:100]
    return {"workload": ("planted KB with the single-hypothesis workload's distributions, N=" + f"{cfg.n:,}"
                         + f"; {n_train:,} engine-scored training hypotheses; 65,536 candidates, top 5 % scored"),
            "n": cfg.n, "n_train": n_train,
            "kb_gen_s": gen_s, "train_scoring_s": score_s, "train_s": train_s, "train_loss": [losses[0], losses[-1]],
            "recall_at_100": OS.recall_at(100, order, sel), "recall_strict_top100": OS.recall_at(100, order, top_pred),
            "selected": k, "best_found": found, "best_acc": float(exact[best, 0]),
            "best_found_per_s": (1.0 / sur_s) if found else 0.0, "best_found_per_s_plain": 1.0 / plain_s,
            "surrogate_round_s": sur_s, "plain_time_to_best_s": plain_s, "mlp_forward": fwd}


def _planner_times(H, handle, batch, reps: int = 5):
    """Time to plan one batch without sharing or bit slicing: the host planner, the
    per-hypothesis planner on 1 and on all host threads, and the device planner from programs
    already in device memory (wall clock including its two synchronisations; best of `reps`;
    the plans are equal, the device image is compared with the host's)."""
    F = H.HEDL_NO_CSE | H.HEDL_NO_SLICE
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def best(fn):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return 1000 * min(ts)

    import torch
    flat, offs = batch
    pd = torch.from_numpy(np.ascontiguousarray(flat).view(np.int64)).cuda()
    od = torch.from_numpy(np.ascontiguousarray(offs, np.uint32).view(np.int32)).cuda()
    host = H.hedl_plan_batch(handle, *batch, F)
    dev = H.hedl_plan_batch_device(handle, pd, od, int(offs[-1]))
    same = bool(np.array_equal(H.hedl_plan_image(host), H.hedl_plan_image(dev)))
    return {"host": best(lambda: H.hedl_plan_batch(handle, *batch, F)),
            "parallel_1": best(lambda: H.hedl_plan_batch_parallel(handle, *batch, F, 1)),
            f"parallel_{cores}": best(lambda: H.hedl_plan_batch_parallel(handle, *batch, F, cores)),
            "device": best(lambda: H.hedl_plan_batch_device(handle, pd, od, int(offs[-1]))),
            "device_image_equals_host": same}


def _section(fn, *a):
    """A secondary workload of the JSON line; a Python-level failure in it is reported in its
    object (with the traceback on stderr) instead of losing the headline line."""
    try:
        return fn(*a)
    except Exception as e:                     # noqa: BLE001 (reported, not hidden)
        import traceback
        traceback.print_exc()
        return {"error": f"{type(e).__name__}: {e}"}


def _oracle_rate(kb, progs, budget_s: float = 6.0):
    """The oracle (as it stands) on the same restrictions, hypothesis-parallel on the host cores,
    for about budget_s seconds; the KB's conversion to the oracle's layout is not timed."""
    import oracle
    from synth import programs as P
    okb = oracle.from_synth(kb)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    done, t0 = 0, time.perf_counter()
    while done < len(progs) and time.perf_counter() - t0 < budget_s:
        sub = progs[done:done + cores]
        oracle.eval_batch(okb, *P.pack_batch(sub), threads=cores)
        done += len(sub)
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "restrictions/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {done} of these restrictions on {cores} host threads ({dt:.1f} s)"}


def _timed_restrictions(dkb, progs, flags, dev, peak, reps=7, label=None):
    """One launch of a batch of restrictions, device-resident: median of `reps` CUDA-event timings on
    the launching stream after warm-up (the graph is captured on the second execution).  The timed
    launches sit in the NVTX range `label`, if given, so a profiler can capture only those."""
    import torch
    import paper_2412_00802_gb300 as H
    from synth import programs as P
    stream = torch.cuda.current_stream(dev)
    flat, offs = P.pack_batch(progs)
    plan = H.hedl_plan_batch(dkb.handle, flat, offs, flags)
    info = H.hedl_plan_info_get(plan)
    ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device=dev)
    counts = torch.zeros((len(progs), 4), dtype=torch.int32, device=dev)
    run = (lambda: H.hedl_plan_execute(dkb.handle, plan, counts, None, ws)) if flags & H.HEDL_PLAIN else \
        (lambda: H.hedl_plan_replay(dkb.handle, plan, counts, None, ws))
    H.hedl_plan_execute(dkb.handle, plan, counts, None, ws)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    ms = []
    if label:
        torch.cuda.nvtx.range_push(label)
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    if label:
        torch.cuda.nvtx.range_pop()
    H.hedl_sync_status(dkb.handle)
    t = statistics.median(ms) / 1000.0
    return {"restrictions": len(progs), "ms": 1000 * t, "restrictions_per_s": len(progs) / t,
            "model_bytes": info["model_bytes"], "achieved_gbs": info["model_bytes"] / t / 1e9,
            "frac": info["model_bytes"] / t / 1e9 / peak}, counts.cpu()


def numeric_run(args, dev):
    """Numeric concrete roles (several values per subject, Section III-B; existential compare,
    Algorithms 9-10) on their own KB: 10^7 individuals, 8 roles of ~4 * 10^7 values U[0, 1000]
    (200 MB of row pointers and values each).  Timed device-resident with CUDA events on the
    launching stream: (a) one >= restriction per role in one interpreter launch (no two read the
    same arrays: 1.6 GB, larger than L2, so every byte comes from HBM), (b) >=, <= and == on every
    role (24 restrictions, one launch), (c) the 24 on the plain path (one launch each)."""
    import torch
    import paper_2412_00802_gb300 as H
    from synth import kb as K, programs as P
    t0 = time.perf_counter()
    kb = K.generate(K.CONFIGS["numeric"])
    gen_s = time.perf_counter() - t0
    dkb = H.DeviceKB.from_synth(kb, device=str(dev))
    peak, kind = measured_peaks()
    thr = [float(v[(q * 7919) % v.size]) for q, v in enumerate(kb.num_vals)]
    one = [np.array([P.insn(P.DGE, 0, q, P.f32_bits(thr[q]))], np.uint64) for q in range(kb.n_num_roles)]
    three = [np.array([P.insn(op, 0, q, P.f32_bits(thr[q]))], np.uint64)
             for q in range(kb.n_num_roles) for op in (P.DGE, P.DLE, P.DEQ)]
    with ClockSampler(dev.index or 0) as clk:
        a, _ = _timed_restrictions(dkb, one, 0, dev, peak, label="numeric_one")
        b, cb = _timed_restrictions(dkb, three, 0, dev, peak, label="numeric_three")
        c, cp = _timed_restrictions(dkb, three, H.HEDL_PLAIN, dev, peak, label="numeric_three_plain")
    # the oracle on roles 0 and 1 (their 6 restrictions), converted alone to keep the run short
    cpu = _oracle_rate(dc_replace(kb, num_row_ptr=kb.num_row_ptr[:2], num_vals=kb.num_vals[:2]), three[:6])
    return {"workload": "N=10,000,000 individuals, 8 numeric concrete roles, Poisson(4) values per individual "
                        "U[0,1000] (~4*10^7 values, 200 MB per role)", "kb_gen_s": gen_s, "cpu_baseline": cpu,
            "values": [int(v.size) for v in kb.num_vals], "kernel": "exec_kernel (exist_words)",
            "peak": peak, "peak_kind": f"{kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "one_per_role": a, "three_per_role": b, "plain_three_per_role": c,
            "plain_counts_identical": bool(torch.equal(cb, cp)), "clocks": clk.summary()}


def string_run(args, dev):
    """String concrete roles (Section III-B; EQUAL, Algorithms 11-12, CONTAIN, Algorithms 13-14) on
    their own KB: 10^7 individuals, 8 roles of ~2 * 10^7 interned ids (120 MB of row pointers and
    ids each) into 100,000 distinct strings, 64 patterns.  Timed like the numeric roles: (a) one
    EQUAL per role (no two read the same arrays: 0.96 GB > L2), (b) EQUAL and CONTAIN of two
    patterns on every role (24 restrictions), (c) the 24 on the plain path.  Load time includes the
    pattern-containment bitmap (64 x 100,000 strings)."""
    import torch
    import paper_2412_00802_gb300 as H
    from synth import kb as K, programs as P
    t0 = time.perf_counter()
    kb = K.generate(K.CONFIGS["strings"])
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dkb = H.DeviceKB.from_synth(kb, device=str(dev))
    load_s = time.perf_counter() - t0
    peak, kind = measured_peaks()
    sid = [int(v[(q * 7919) % v.size]) for q, v in enumerate(kb.str_ids)]
    one = [np.array([P.insn(P.SEQ, 0, q, sid[q])], np.uint64) for q in range(kb.n_str_roles)]
    mixed = []
    for q in range(kb.n_str_roles):
        mixed += [np.array([P.insn(P.SEQ, 0, q, sid[q])], np.uint64),
                  np.array([P.insn(P.SCONTAINS, 0, q, 1 + q)], np.uint64),
                  np.array([P.insn(P.SCONTAINS, 0, q, 17 + q)], np.uint64)]
    with ClockSampler(dev.index or 0) as clk:
        a, _ = _timed_restrictions(dkb, one, 0, dev, peak, label="strings_one")
        b, cb = _timed_restrictions(dkb, mixed, 0, dev, peak, label="strings_mixed")
        c, cp = _timed_restrictions(dkb, mixed, H.HEDL_PLAIN, dev, peak, label="strings_mixed_plain")
    cpu = _oracle_rate(dc_replace(kb, str_row_ptr=kb.str_row_ptr[:2], str_ids=kb.str_ids[:2]), mixed[:6])
    return {"workload": "N=10,000,000 individuals, 8 string concrete roles, Poisson(2) values per individual "
                        "(~2*10^7 ids, 120 MB per role) into 100,000 distinct strings of 3-12 letters; 64 "
                        "patterns", "kb_gen_s": gen_s, "kb_load_s_with_bitmap": load_s, "cpu_baseline": cpu,
            "values": [int(v.size) for v in kb.str_ids], "kernel": "exec_kernel (exist_words)",
            "peak": peak, "peak_kind": f"{kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "equal_one_per_role": a, "equal_and_contain": b, "plain_equal_and_contain": c,
            "plain_counts_identical": bool(torch.equal(cb, cp)), "clocks": clk.summary()}


def search_run(args, dev):
    """The refinement beam search on a planted KB with the search workload's distributions:
    exhaustive (every candidate scored) against surrogate-ordered with pruning."""
    import torch
    import paper_2412_00802_gb300 as H
    from paper_2412_00802_gb300.search import BeamSearch
    from paper_2412_00802_gb300.surrogate import Surrogate, exact_scores
    from synth import hyps, kb as K, programs as P
    from synth.refine import Refiner
    full = not args.search_small
    cfg = K.CONFIGS["search"] if full else K.CONFIGS["search"].scaled(1_000_000)
    t0 = time.perf_counter()
    kb = K.generate(cfg)
    gen_s = time.perf_counter() - t0
    dkb = H.DeviceKB.from_synth(kb, device=str(dev))
    ref = Refiner(kb, 505)

    def refine(beam_progs, step, count):
        return ref.refine_postfix(beam_progs, step, count)
    start = [np.array(n.postfix(), np.uint64) for n in ref.start()]
    steps = 20 if full else 10
    from paper_2412_00802_gb300.surrogate import threshold_grid
    sur = Surrogate(seed=5, device=str(dev), grid=threshold_grid(kb.prop_vals))
    sur.fit_statistics(dkb, kb.n_concepts)
    tg = hyps.TreeGen(kb, 506, share=0.3)
    Xs, Ts = [], []
    for b in range(8):
        flat, offs = _pack(hyps.batch_hyps(kb, 506, b, 4096, gen=tg))
        _, T = exact_scores(dkb, flat, offs)
        Xs.append(sur.encode(flat, offs))
        Ts.append(T)
    sur.train(torch.cat(Xs), torch.cat(Ts), epochs=40, batch=4096, lr=2e-3)
    out = {"workload": f"planted KB with the search workload's distributions, N={cfg.n:,}, {kb.n_roles} roles; "
                       f"beam 64, 8,192 refinements per step, {steps} steps", "kb_gen_s": gen_s,
           "n": cfg.n, "steps": steps}
    res = {}
    state, tmap = sur.params().copy(), sur.target_map()
    online = {"online_epochs": 2, "online_window": 16384}
    variants = (("exhaustive", {}, 2048),
                ("surrogate_ordered", dict(online), 2048),
                ("surrogate_pruned", dict(online, keep_fraction=0.25, warmup_steps=1), 2048),
                ("surrogate_adaptive", dict(online, adaptive=True, warmup_steps=1), 1024))
    for name, kw, batch in variants:
        if "online_epochs" in kw:     # each surrogate run starts from the same pre-trained network
            net = Surrogate(params=state, device=str(dev), grid=threshold_grid(kb.prop_vals))
            net.set_target_map(tmap)
            net.stats, net.n_stat_concepts = sur.stats, sur.n_stat_concepts
            kw = dict(kw, surrogate=net)
        t0 = time.perf_counter()
        beam, logs = BeamSearch(dkb, refine, width=64, per_step=8192, batch=batch, **kw).run(start, steps)
        res[name] = (beam, logs, time.perf_counter() - t0)
    eb = res["exhaustive"][0]
    target = eb[0].acc

    def first_reach(logs):
        for l in logs:
            for t, b in l.events:
                if b >= target:
                    return t
        return None
    out["best_acc"] = target
    out["best"] = P.to_text(P.from_postfix(eb[0].prog))
    for name, (beam, logs, secs) in res.items():
        t = first_reach(logs)
        out[name] = {"seconds": secs, "best_acc": beam[0].acc, "evaluated": sum(l.evaluated for l in logs),
                     "candidates": sum(l.candidates for l in logs),
                     "best_found_per_s": 1.0 / t if t else 0.0,
                     "same_final_beam": [e.prog.tobytes() for e in beam] == [e.prog.tobytes() for e in eb],
                     "seconds_by_part": {k: round(sum(l.times.get(k, 0.0) for l in logs), 4)
                                         for k in ("refine", "surrogate", "eval", "learn")}}
    return out


def latency_measure(args, dev, tune: bool = True):
    """Single large hypothesis latency: the 10,000,000-individual KB (32 Zipf(2.1) roles,
    ~2.6 G assertions), 64 depth-6 hypotheses with chains of 3 nested EXISTS / ATLEAST,
    each evaluated alone through hedl_eval_concept (plan + upload + launch) and timed with
    CUDA events; algorithmic bytes per hypothesis from its plan."""
    import torch
    import paper_2412_00802_gb300 as H
    from synth import hyps, kb as K, programs as P
    t0 = time.perf_counter()
    cfg = K.CONFIGS["large"]
    if args.latency_n:                       # smaller KB of the same distributions (profiling)
        cfg = cfg.scaled(args.latency_n)
    kb = K.generate(cfg)
    gen_s = time.perf_counter() - t0
    dkb = H.DeviceKB.from_synth(kb, device=str(dev))
    progs = hyps.chain_hyps(kb, 2002, 64)
    tune_s = None
    if tune:
        # launch shape picked on another hypothesis of the same shape, evaluated alone
        t0 = time.perf_counter()
        dkb.autotune(*P.pack_batch(hyps.chain_hyps(kb, 2003, 1)))
        tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    out = torch.zeros(dkb.wp, dtype=torch.int32, device=dev)
    for p in progs[:3]:                       # warm-up
        dkb.eval(p, args.flags)
    lat, model, host, replay, levels = [], [], [], [], []
    offs = lambda p: np.array([0, len(p)], np.uint32)
    with ClockSampler(dev.index or 0) as clk:
        for p in progs:
            nbytes = H.hedl_workspace_size(dkb.handle, p, offs(p), args.flags)
            ws = dkb.workspace(nbytes)
            plan = H.hedl_plan_batch(dkb.handle, p, offs(p), args.flags)
            info = H.hedl_plan_info_get(plan)
            model.append(info["model_bytes"])
            levels.append(info["n_levels"])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            h0 = time.perf_counter()
            H.hedl_eval_concept(dkb.handle, p, out, ws, args.flags)
            host.append(time.perf_counter() - h0)
            b.record(stream)
            torch.cuda.synchronize()
            lat.append(a.elapsed_time(b) / 1000.0)
            # the same plan again, resident: device time without planning and upload
            H.hedl_plan_execute(dkb.handle, plan, None, out, ws)
            H.hedl_plan_replay(dkb.handle, plan, None, out, ws)
            torch.cuda.synchronize()
            a.record(stream)
            H.hedl_plan_replay(dkb.handle, plan, None, out, ws)
            b.record(stream)
            torch.cuda.synchronize()
            replay.append(a.elapsed_time(b) / 1000.0)
    H.hedl_sync_status(dkb.handle)
    peak, kind = measured_peaks()
    gbs = [m / t / 1e9 for m, t in zip(model, lat)]
    res = {
        "workload": "N=10,000,000 individuals, 200 concepts, 32 roles Zipf(2.1) mean 8 cap 10^4 + inverses, "
                    "16 props lognormal(0,1) 10% missing, 100k/100k examples; 64 depth-6 hypotheses with "
                    "3-chains of EXISTS/ATLEAST, one at a time",
        "n": kb.n, "kb_gen_s": gen_s, "flags": args.flags, "tuning": H.hedl_tuning_get(dkb.handle),
        "autotune_s": tune_s,
        "latency_ms": {"median": 1000 * statistics.median(lat), "min": 1000 * min(lat), "max": 1000 * max(lat),
                       "host_call_median": 1000 * statistics.median(host),
                       "resident_replay_median": 1000 * statistics.median(replay)},
        "levels_median": statistics.median(levels),
        "model": {"achieved_gbs": statistics.median(gbs), "peak": peak, "frac": statistics.median(gbs) / peak,
                  "peak_kind": f"{kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                  "model_bytes_median": statistics.median(model)},
        "clocks": clk.summary()}
    del dkb
    torch.cuda.empty_cache()
    return res


def run_latency(args, local_rank):
    """The single-hypothesis latency workload alone (one JSON line, time-like metric)."""
    import torch
    from paper_2412_00802_gb300 import build
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    build.build()
    r = latency_measure(args, dev, tune=not args.no_tune)
    print(json.dumps({
        "metric": "single-hypothesis latency", "value": r["latency_ms"]["median"], "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": 64, "dtype": "u32", "data": "synthetic",
        "config": {"workload": r["workload"], "kb_gen_s": r["kb_gen_s"], "n": r["n"], "flags": r["flags"],
                   "tuning": r["tuning"], "autotune_s": r["autotune_s"]},
        "latency_ms": r["latency_ms"], "levels_median": r["levels_median"],
        "roofline": {"bound": "hbm", "achieved": r["model"]["achieved_gbs"], "peak": r["model"]["peak"],
                     "unit": "GB/s", "frac": r["model"]["frac"], "traffic": None,
                     "peak_kind": r["model"]["peak_kind"], "model_bytes_median": r["model"]["model_bytes_median"],
                     "note": "algorithmic bytes of the plan (byte model) / CUDA-event latency"},
        "clocks": r["clocks"]}), flush=True)


def run_mlp(args, local_rank):
    """The surrogate's forward alone: 65,536 encoded random hypotheses (a 20,000-individual KB
    of the surrogate workload's distributions) through both GEMM engines."""
    import torch
    from paper_2412_00802_gb300 import build
    from paper_2412_00802_gb300 import surrogate as sg
    from synth import hyps, kb as K, programs as P
    torch.cuda.set_device(local_rank)
    build.build()
    kb = K.generate(K.CONFIGS["surrogate"].scaled(20_000))
    progs = hyps.batch_hyps(kb, 77, 0, 65_536, gen=hyps.TreeGen(kb, 77, share=0.3))
    s = sg.Surrogate(seed=1, device=f"cuda:{local_rank}", grid=sg.threshold_grid(kb.prop_vals))
    X = s.encode(*P.pack_batch(progs))
    fwd = mlp_forward_timing(s, X)
    print(json.dumps({"metric": "surrogate forward TFLOP/s (tcgen05)", "value": fwd["tcgen05"]["tflops"],
                      "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1, "dtype": "bf16",
                      "data": "synthetic", "config": {"workload": "MLP 512-512-512-2 forward, 65,536 rows"},
                      "mlp_forward": fwd}), flush=True)


def run_reference(args, rank, world):
    """Reference arm: the oracle timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    kb = make_workload()
    from synth import hyps
    gen = hyps.TreeGen(kb, 1003, share=0.3)
    import oracle
    from synth import programs as P
    okb = oracle.from_synth(kb)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    per_step = max(cores, 16)
    steps = []
    for s in range(args.warmup + args.steps):
        progs = make_batch(kb, s, gen)[:per_step]
        flat, offs = P.pack_batch(progs)
        t0 = time.perf_counter()
        oracle.eval_batch(okb, flat, offs, threads=cores)
        steps.append(time.perf_counter() - t0)
    timed = steps[args.warmup:]
    value = per_step * len(timed) / sum(timed)
    sample = f"{per_step} hypotheses per step (of each 4,096-hypothesis batch), {cores} host threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(timed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "parallelism": "replicas1", "sample_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2412_00802_gb300 as H
    from paper_2412_00802_gb300 import build
    from synth import hyps, programs as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    build.build()
    kb = make_workload()
    dkb = H.DeviceKB.from_synth(kb, device=f"cuda:{local_rank}")
    gen = hyps.TreeGen(kb, 1003, share=0.3)
    warm_ids, timed_ids = shard_batches(rank, world, args.warmup, args.steps)
    ids = warm_ids + timed_ids
    if args.one_batch:            # profiling: every step replays the first timed batch on one workspace
        one = P.pack_batch(make_batch(kb, timed_ids[0], gen))
        batches = {i: one for i in ids}
    else:
        batches = {i: P.pack_batch(make_batch(kb, i, gen)) for i in ids}
    tune_s = None
    if not args.no_tune:
        # launch shape picked by the autotuner on a probe batch (not a timed one)
        probe = P.pack_batch(make_batch(kb, 10_000 + rank, gen, count=512))
        t0 = time.perf_counter()
        dkb.autotune(*probe)
        tune_s = time.perf_counter() - t0

    stream = torch.cuda.current_stream(dev)
    # ---- plan every batch (host), give each its own workspace, upload once
    plans, infos, wss = {}, {}, {}
    plan_s = []
    for i in ids:
        if args.one_batch and i != ids[0]:
            plans[i], infos[i], wss[i] = plans[ids[0]], infos[ids[0]], wss[ids[0]]
            continue
        t0 = time.perf_counter()
        plans[i] = H.hedl_plan_batch(dkb.handle, *batches[i], args.flags)
        plan_s.append(time.perf_counter() - t0)
        infos[i] = H.hedl_plan_info_get(plans[i])
        wss[i] = torch.empty(infos[i]["workspace_bytes"], dtype=torch.uint8, device=dev)
    counts = torch.zeros((BATCH, 4), dtype=torch.int32, device=dev)
    for i in (ids[:1] if args.one_batch else ids):
        H.hedl_plan_execute(dkb.handle, plans[i], counts, None, wss[i])
    H.hedl_sync_status(dkb.handle)
    for i in timed_ids:          # second execution: the plan's CUDA graph is captured here
        H.hedl_plan_replay(dkb.handle, plans[i], counts, None, wss[i])
    for i in warm_ids:
        H.hedl_plan_replay(dkb.handle, plans[i], counts, None, wss[i])
    H.hedl_sync_status(dkb.handle)

    # ---- timed region: device-resident replays, events per launch on the launching stream
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in timed_ids]
    with ClockSampler(local_rank) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")    # lets a profiler capture only these launches
        t_all0.record(stream)
        for (a, b), i in zip(ev, timed_ids):
            a.record(stream)
            H.hedl_plan_replay(dkb.handle, plans[i], counts, None, wss[i])
            b.record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    H.hedl_sync_status(dkb.handle)
    elapsed = t_all0.elapsed_time(t_all1) / 1000.0
    if dist:
        elapsed = max_over_ranks(elapsed, dev)
        torch.distributed.barrier()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    value = world * len(timed_ids) * BATCH / elapsed

    # ---- roofline of the interpreter launch.  The kernel is timed by CUDA events on its stream;
    # its DRAM bytes per launch come from the committed ncu capture of the same interpreter code
    # and launch shape (profiles/traffic.json), so `achieved` is measured HBM traffic / time.  The
    # plan's algorithmic bytes (the per-operation byte model, what the plain method would move)
    # over the same time are the "effective" figure: far above the peak, since bit-sliced walks and
    # L2 reuse read each role's arrays once for many restrictions.
    peak, peak_kind = measured_peaks()
    model = [infos[i]["model_bytes"] for i in timed_ids]
    launch_s = statistics.mean(launch_ms) / 1000.0
    effective = statistics.mean(m / (t / 1000.0) for m, t in zip(model, launch_ms)) / 1e9
    tuning_now = H.hedl_tuning_get(dkb.handle)
    prof = traffic_for("batch", tuning_now)
    traffic = prof["dram_bytes_per_launch"] if prof else None
    achieved = traffic / launch_s / 1e9 if traffic else None
    l2_frac = prof.get("lts_throughput_pct", None) if prof else None

    # ---- end to end through the public C ABI from host programs: each step plans a batch
    # on the host (hedl_plan_batch), uploads and launches it (hedl_plan_execute) and copies
    # its counts to pinned host memory; the next batch is planned while the GPU runs this one
    e2e_ids = timed_ids[: min(len(timed_ids), 8)]
    pinned = [torch.empty((BATCH, 4), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    wsz = max(infos[i]["workspace_bytes"] for i in ids)
    e2e_ws = [torch.empty(wsz, dtype=torch.uint8, device=dev) for _ in range(2)]
    e2e_counts = [torch.zeros((BATCH, 4), dtype=torch.int32, device=dev) for _ in range(2)]
    done_ev = [torch.cuda.Event(), torch.cuda.Event()]
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    h2d = []
    t0 = time.perf_counter()
    plan = H.hedl_plan_batch(dkb.handle, *batches[e2e_ids[0]], args.flags)
    held = [None, None]
    for q, i in enumerate(e2e_ids):
        b = q & 1
        H.hedl_plan_execute(dkb.handle, plan, e2e_counts[b], None, e2e_ws[b])
        pinned[b].copy_(e2e_counts[b], non_blocking=True)
        done_ev[b].record(stream)
        h2d.append(H.hedl_plan_info_get(plan)["image_bytes"])
        held[b] = plan                                   # keep the plan alive until its step is done
        if q + 1 < len(e2e_ids):
            plan = H.hedl_plan_batch(dkb.handle, *batches[e2e_ids[q + 1]], args.flags)
        if q >= 1:
            done_ev[1 - b].synchronize()                  # the previous step's counts are on the host
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:                                              # whole job: every rank's batches, slowest rank
        e2e_s = max_over_ranks(e2e_s, dev)
    H.hedl_sync_status(dkb.handle)
    e2e = {"value": world * len(e2e_ids) * BATCH / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(statistics.mean(h2d)), "d2h_bytes_per_step": BATCH * 16,
           "note": "host programs -> hedl_plan_batch -> hedl_plan_execute (plan upload + launch) -> counts to "
                   "pinned host memory, wall clock; the next batch is planned while the GPU runs the current one"}
    del e2e_ws
    torch.cuda.empty_cache()

    # ---- plain path (one launch per operation) on the first timed batch, and sharing off
    plain = None
    if not args.no_plain:
        i = timed_ids[0]
        pplan = H.hedl_plan_batch(dkb.handle, *batches[i], H.HEDL_PLAIN)
        pws = torch.empty(H.hedl_plan_info_get(pplan)["workspace_bytes"], dtype=torch.uint8, device=dev)
        pcounts = torch.zeros((BATCH, 4), dtype=torch.int32, device=dev)
        H.hedl_plan_execute(dkb.handle, pplan, pcounts, None, pws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        H.hedl_plan_execute(dkb.handle, pplan, pcounts, None, pws)
        b.record(stream)
        torch.cuda.synchronize()
        H.hedl_sync_status(dkb.handle)
        plain = {"value": BATCH / (a.elapsed_time(b) / 1000.0), "unit": UNIT}
        # verify the batched counts of that batch against the plain path
        H.hedl_plan_replay(dkb.handle, plans[i], counts, None, wss[i])
        torch.cuda.synchronize()
        plain["counts_identical"] = bool(torch.equal(pcounts, counts))
    info0 = infos[timed_ids[0]]
    ncse = H.hedl_plan_info_get(H.hedl_plan_batch(dkb.handle, *batches[timed_ids[0]], H.HEDL_NO_CSE))
    planners = _section(_planner_times, H, dkb.handle, batches[timed_ids[0]])

    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline(kb, make_batch(kb, timed_ids[0], gen))
    clocks = clk.summary()
    # the secondary workloads run on KBs of their own: free this one's device memory first
    del wss, dkb
    torch.cuda.empty_cache()
    latency = None if args.no_latency else _section(latency_measure, args, dev, not args.no_tune)
    surrogate = None if args.no_surrogate else _section(surrogate_round, args, dev)
    search = None if args.no_search else _section(search_run, args, dev)
    numeric = None if args.no_numeric else _section(numeric_run, args, dev)
    strings = None if args.no_strings else _section(string_run, args, dev)
    plan_info = {"host_ms_per_batch": 1000 * statistics.mean(plan_s), "segments": info0["n_segments"],
                 "slots": info0["n_slots"], "levels": info0["n_levels"], "items": info0["n_items"],
                 "role_ops": info0["n_role_ops"], "role_groups": info0["n_role_groups"],
                 "role_ops_without_sharing": ncse["n_role_ops"],
                 "model_bytes": info0["model_bytes"], "model_bytes_without_sharing": ncse["model_bytes"],
                 "no_sharing_planners_ms": planners}
    details = {"plain": plain, "plan": plan_info, "latency": latency, "surrogate": surrogate, "search": search,
               "numeric_roles": numeric, "string_roles": strings,
               "cpu_single_thread": cpu.get("single_thread") if cpu else None}
    # every secondary workload in full, on one stderr line (the stdout line stays short)
    print(json.dumps({"details": details}), file=sys.stderr, flush=True)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(timed_ids),
        "warmup": len(warm_ids), "ms_per_step": 1000.0 * elapsed / len(timed_ids), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "l2": "inputs larger than L2 (KB ~0.95 GB + workspaces)",
                   "parallelism": f"replicas{world}", "flags": args.flags, "one_batch": bool(args.one_batch),
                   "tuning": tuning_now, "autotune_s": tune_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "l2_frac": l2_frac,
                     "effective_gbs": effective, "effective_frac": effective / peak,
                     "algorithmic_bytes_per_launch": statistics.mean(model),
                     "launch_ms": statistics.mean(launch_ms),
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": "exec_kernel (persistent segment interpreter)",
                     "note": "achieved = ncu DRAM bytes per launch (traffic) / CUDA-event launch time; "
                             "effective = the plan's algorithmic bytes / the same time"},
        "cpu_baseline": {k: v for k, v in cpu.items() if k != "single_thread"} if cpu else None,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": 2 * len(timed_ids),
        "secondary": _summary(value / world, plain, plan_info, ncse, peak, latency, surrogate, search, numeric,
                              strings, cpu),
    }
    print(json.dumps(out), flush=True)


def run_scheduled(args, rank, world, local_rank):
    """The batched workload with every step's global batch (world x 4,096 hypotheses) split
    across the ranks by the paper's probe-timed static ratios (--schedule static) or handed out
    in chunks by a host work queue in the process group's store (--schedule dynamic); see
    paper_2412_00802_gb300/schedule.py.  Shares are planned and executed from host programs
    inside the timed region (plan, upload, launch, counts back), the counts of every step are
    gathered and checked to cover each hypothesis once.  value = all ranks' hypotheses / the
    slowest rank's time."""
    import torch
    import torch.distributed as td
    import paper_2412_00802_gb300 as H
    from paper_2412_00802_gb300 import build, schedule as SC
    from synth import hyps, programs as P
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    build.build()
    kb = make_workload()
    dkb = H.DeviceKB.from_synth(kb, device=f"cuda:{local_rank}")
    gen = hyps.TreeGen(kb, 1003, share=0.3)
    Hg = world * BATCH
    steps = list(range(args.warmup + args.steps))
    batches = {s: make_batch(kb, 50_000 + s, gen, count=Hg) for s in steps}
    dist = world > 1
    probe = SC.probe_program(kb.n_concepts)
    out = torch.zeros(dkb.wp, dtype=torch.int32, device=dev)
    pws = dkb.workspace(H.hedl_workspace_size(dkb.handle, probe, np.array([0, len(probe)], np.uint32)))

    def run_probe():
        H.hedl_eval_concept(dkb.handle, probe, out, pws)
        torch.cuda.synchronize()
    rates = SC.probe_rates(run_probe, reps=20, warmup=3)
    store = td.distributed_c10d._get_default_store() if dist else td.HashStore()
    chunk = 1024
    wsz = max(H.hedl_workspace_size(dkb.handle, *P.pack_batch(batches[steps[0]][i:i + chunk]))
              for i in range(0, Hg, chunk))
    ws = dkb.workspace(2 * wsz)
    counts = torch.zeros((max(chunk, Hg), 4), dtype=torch.int32, device=dev)

    def do_share(progs):
        flat, offs = P.pack_batch(progs)
        plan = H.hedl_plan_batch(dkb.handle, flat, offs)
        c = counts[:len(progs)]
        H.hedl_plan_execute(dkb.handle, plan, c, None, ws)
        return c.cpu().numpy()

    def step(s):
        progs = batches[s]
        idx, got = [], []
        if args.schedule == "static":
            b, e = SC.split_by_rates(rates, Hg, 64)[rank]
            for i in range(b, e, chunk):
                idx.append(np.arange(i, min(e, i + chunk)))
                got.append(do_share(progs[i:min(e, i + chunk)]))
        else:
            q = SC.DynamicQueue(store, f"bench{s}", Hg, chunk)
            while (r := q.next()) is not None:
                idx.append(np.arange(*r))
                got.append(do_share(progs[r[0]:r[1]]))
        return (np.concatenate(idx) if idx else np.zeros(0, np.int64),
                np.concatenate(got) if got else np.zeros((0, 4), np.int64), len(np.concatenate(idx)) if idx else 0)

    for s in steps[:args.warmup]:
        step(s)
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    mine, kept = 0, []
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        for s in steps[args.warmup:]:
            i, c, k = step(s)
            kept.append((i, c))
            mine += k
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
    if dist:
        elapsed = max_over_ranks(elapsed, dev)
    for i, c in kept:                         # every hypothesis of every step scored exactly once
        SC.gather_counts(i, c, Hg, dst=0)
    shares = [None] * world
    if dist:
        td.all_gather_object(shares, mine)
    else:
        shares = [mine]
    if rank != 0:
        return
    value = world * BATCH * args.steps / elapsed
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "global_batch": Hg, "schedule": args.schedule,
                   "chunk": chunk, "probe_rates": rates, "hypotheses_per_rank": shares,
                   "parallelism": f"{args.schedule}{world}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": Hg * 16,
                "note": "shares planned, uploaded, launched and read back inside the timed region"},
        "clocks": clk.summary(), "gpu_launches": None}), flush=True)


def _summary(value, plain, plan_info, ncse, peak, latency, surrogate, search, numeric, strings, cpu):
    """The secondary figures, rounded, flat enough to survive a truncated stdout tail."""
    def ok(x):
        return x if isinstance(x, dict) and "error" not in x else None
    out = {"batched_vs_plain": _r(value / plain["value"]) if plain else None,
           "plain_hyp_s": _r(plain["value"]) if plain else None,
           "plain_counts_identical": plain["counts_identical"] if plain else None,
           "effective_frac_unshared": _r(value * (ncse["model_bytes"] / BATCH) / 1e9 / peak),
           "plan_ms": _r(plan_info["host_ms_per_batch"]), "role_ops": plan_info["role_ops"],
           "plan_no_sharing_ms": {k: (_r(v) if not isinstance(v, bool) else v)
                                  for k, v in (plan_info["no_sharing_planners_ms"] or {}).items()
                                  if k != "error"},
           "role_groups": plan_info["role_groups"],
           "cpu_1thread_hyp_s": _r(cpu["single_thread"]["value"]) if cpu else None}
    if ok(latency):
        out["latency"] = {"n": latency["n"], "median_ms": _r(latency["latency_ms"]["median"]),
                          "replay_ms": _r(latency["latency_ms"]["resident_replay_median"]),
                          "model_gbs": _r(latency["model"]["achieved_gbs"]), "model_frac": _r(latency["model"]["frac"])}
    if ok(surrogate):
        f = surrogate["mlp_forward"]
        out["surrogate"] = {"n": surrogate["n"], "train": surrogate["n_train"],
                            "recall_at_100": surrogate["recall_at_100"],
                            "recall_strict": surrogate["recall_strict_top100"], "best_found": surrogate["best_found"],
                            "bfps": _r(surrogate["best_found_per_s"]),
                            "bfps_plain": _r(surrogate["best_found_per_s_plain"]),
                            "mlp_tflops": _r(f["tcgen05"]["tflops"]), "mlp_frac": _r(f["tcgen05"]["frac"]),
                            "mlp_ms_median": _r(f["tcgen05"]["ms"]),
                            "mma_sync_tflops": _r(f["mma_sync"]["tflops"])}
    if ok(search):
        out["search"] = {"n": search["n"], "steps": search["steps"], "best_acc": search["best_acc"]}
        for k in ("exhaustive", "surrogate_pruned", "surrogate_adaptive"):
            if k in search:
                out["search"][k] = {"bfps": _r(search[k]["best_found_per_s"]), "s": _r(search[k]["seconds"]),
                                    "same_beam": search[k]["same_final_beam"]}
    if ok(numeric):
        out["numeric_frac"] = [_r(numeric["one_per_role"]["frac"]), _r(numeric["three_per_role"]["frac"])]
    if ok(strings):
        out["string_frac"] = [_r(strings["equal_one_per_role"]["frac"]), _r(strings["equal_and_contain"]["frac"])]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", type=int, default=0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate-ranked round")
    ap.add_argument("--no-search", action="store_true", help="skip the beam-search comparison")
    ap.add_argument("--no-numeric", action="store_true", help="skip the numeric-concrete-role workload")
    ap.add_argument("--no-strings", action="store_true", help="skip the string-concrete-role workload")
    ap.add_argument("--surrogate-train", type=int, default=0,
                    help="training hypotheses of the surrogate round (default 1,000,000; 65,536 with "
                         "--surrogate-small)")
    ap.add_argument("--surrogate-small", action="store_true",
                    help="surrogate round on a 1M-individual KB of its distributions (the full size is 10M "
                         "individuals and 1M training hypotheses, the default)")
    ap.add_argument("--latency", action="store_true",
                    help="the single-hypothesis latency workload (10M individuals) instead of the batched one")
    ap.add_argument("--mlp", action="store_true", help="time the surrogate's forward alone (both GEMM engines)")
    ap.add_argument("--latency-n", type=int, default=0,
                    help="individuals of the latency workload's KB (default: its full 10,000,000)")
    ap.add_argument("--search-small", action="store_true",
                    help="search on a 1M-individual KB for 10 steps (the full size, 4M individuals and 20 steps, "
                         "is the default)")
    ap.add_argument("--no-latency", action="store_true", help="skip the single-hypothesis latency section")
    ap.add_argument("--schedule", default="replicas", choices=["replicas", "static", "dynamic"],
                    help="replicas: each rank its own batches (default); static: every global batch split by "
                         "the probe-timed ratios; dynamic: chunks from a host work queue")
    ap.add_argument("--one-batch", action="store_true",
                    help="every step replays one batch on one workspace (small device footprint, for ncu)")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="hypotheses per step (smaller only for profiling captures)")
    args = ap.parse_args()
    globals()["BATCH"] = args.batch
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as td
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        td.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.latency:
        run_latency(args, local_rank)
    elif args.mlp:
        run_mlp(args, local_rank)
    elif args.schedule != "replicas":
        run_scheduled(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.barrier()
        td.destroy_process_group()


if __name__ == "__main__":
    main()
