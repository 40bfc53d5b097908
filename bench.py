"""Benchmark of the GB300 parallel-sentence miner.

Default workload: 10,000 synthetic comparable-article pairs with lognormal
sentence counts (median 60, clipped 5-800), 5-40-token sentences over a 200k
Zipf vocabulary and a 200k-entry dictionary, gap -1.0, threshold 0.5 (Q16).

One step = the whole mining path (score matrices, alignments, tracebacks,
selection) over the batch.  `value` is article pairs/s with the batch resident
in device memory; `e2e` is the same through the host-buffer C calls (copies
in and results out inside the timed region, two calls in flight so that one
call's input copies overlap the kernels of the one before; also one call at a
time); `plain` mines one pair per call.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes
import datetime
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "article pairs/s & NW GCUPS, batched/served vs plain per-pair, 1 GB300; p50/p99"
UNIT = "article pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", type=int, default=2, help="1..5 (parity cases); 2 is the bench")
    ap.add_argument("--pairs", type=int, default=None, help="override the pair count")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--plain-pairs", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=5000.0)
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="seconds per offered load (30 s as config 5 states)")
    ap.add_argument("--configs", default="1,3,4",
                    help="other workloads measured after the benchmark batch (sub-records)")
    ap.add_argument("--serve-sweep", default="1000,20000",
                    help="further offered rates (pairs/s), --serve-seconds each; empty for none")
    ap.add_argument("--only-device", action="store_true",
                    help="time only the device-resident path (for profiler captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the bidirectional-mining and tuning-objective measurements")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in alignment strategy (no tuning launches before the run)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(workload: int, rank: int):
    """Seed of the batch a rank mines: rank 0 mines the standard batch, every
    other rank its own independent batch of the same shape (weak scaling)."""
    return None if rank == 0 else 1508 + workload + 1000 * rank


def max_over_ranks(x: float, ws: int) -> float:
    """The slowest rank's value (time-like quantities)."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return ws * units_per_rank / seconds


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region.  Each
    sample carries nvidia-smi's own timestamp; the summary keeps those taken
    between mark_start() and mark_end() (all samples when none was, or when
    the timestamps cannot be read)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 10
    TS_FORMAT = "%Y/%m/%d %H:%M:%S.%f"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @classmethod
    def parse(cls, line):
        """(time or None, sm MHz, max sm MHz, hw, hw thermal, sw thermal, power cap)."""
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            return None
        try:
            row = (float(f[2]), float(f[3]), f[6], f[7], f[8], f[9])
        except ValueError:
            return None
        try:
            t = datetime.datetime.strptime(f[0], cls.TS_FORMAT).timestamp()
        except ValueError:
            t = None
        return (t,) + row

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = [r for r in (self.parse(line) for line in open(self.path)) if r is not None]
        os.unlink(self.path)
        if not rows:
            return None
        window = "whole sampler run"
        if self.t0 is not None and self.t1 is not None and all(r[0] is not None for r in rows):
            inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
            if inside:
                rows, window = inside, "timed region"
        sm = [r[1] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": reasons, "samples": len(rows), "window": window,
                "interval_ms": self.INTERVAL_MS}


# --------------------------------------------------------------------- helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "align.cu", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1509_08639_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch from a committed ncu summary, when it still
    describes the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    k = d.get("kernels", {}).get(kernel)
    if not k or d.get("source_hash") != kernel_source_hash():
        return None
    return k.get("dram_bytes_per_launch_full_workload")


def _sorted_unique(x):
    y = np.sort(x)
    return y[np.concatenate(([True], y[1:] != y[:-1]))] if y.shape[0] else y


def kept_entries(w):
    """Entries the preparation kernel writes: over every source sentence's
    distinct tokens, their dictionary translations that the pair's target
    article holds (numpy, from the inputs alone)."""
    b, d = w.batch, w.dictionary
    doc = b.doc_off.astype(np.int64)
    so = b.sent_off.astype(np.int64)
    n_sent = so.shape[0] - 1
    sent_doc = np.repeat(np.arange(doc.shape[0] - 1, dtype=np.int64), np.diff(doc))
    tok_sent = np.repeat(np.arange(n_sent, dtype=np.int64), np.diff(so))
    tok_doc = sent_doc[tok_sent]
    tokens = b.tokens.astype(np.int64)
    tgt = (tok_doc & 1) == 1
    tgt_keys = _sorted_unique(((tok_doc[tgt] >> 1) << 32) | tokens[tgt])
    st = _sorted_unique((tok_sent[~tgt] << 32) | tokens[~tgt])
    s_sent, s_tok = st >> 32, st & 0xFFFFFFFF
    keys = d.keys.astype(np.int64)
    if keys.shape[0] == 0:
        return 0
    toff = d.trans_off.astype(np.int64)
    order = np.argsort(keys)
    ks = keys[order]
    pos = np.minimum(np.searchsorted(ks, s_tok), ks.shape[0] - 1)
    found = ks[pos] == s_tok
    kidx = order[pos[found]]
    off, cnt = toff[kidx], toff[kidx + 1] - toff[kidx]
    first = np.cumsum(cnt) - cnt
    idx = np.repeat(off - first, cnt) + np.arange(int(cnt.sum()), dtype=np.int64)
    u = d.trans.astype(np.int64)[idx]
    upair = sent_doc[np.repeat(s_sent[found], cnt)] >> 1
    q = (upair << 32) | u
    at = np.minimum(np.searchsorted(tgt_keys, q), tgt_keys.shape[0] - 1)
    return int((tgt_keys[at] == q).sum()) if tgt_keys.shape[0] else 0


def cpu_baseline(w, budget_s=20.0):
    """The oracle as it stands, on this host's cores, on a bounded sample."""
    from oracle import oracle as O
    od = O.OracleDict(w.dictionary)
    S, T = w.batch.sizes()
    rng = np.random.default_rng(99)
    order = rng.permutation(w.batch.n_pairs)
    threads = os.cpu_count() or 1
    done_pairs, done_cells, t_used, k = 0, 0, 0.0, 0
    chunk = max(threads * 4, 32)
    while t_used < budget_s and k < len(order):
        idx = order[k:k + chunk]
        sub = w.batch.subset(idx)
        t0 = time.perf_counter()
        _, used = O.mine_batch(od, sub, w.settings, threads)
        t_used += time.perf_counter() - t0
        done_pairs += len(idx)
        done_cells += int((S[idx] * T[idx]).sum())
        k += chunk
    # the same oracle on one core, on a shorter sample
    one_pairs, one_t, k1 = 0, 0.0, 0
    one_order = rng.permutation(w.batch.n_pairs)
    while one_t < budget_s / 4 and k1 < len(one_order):
        idx = one_order[k1:k1 + 1]   # one pair at a time: a sample ends within one pair of its budget
        t0 = time.perf_counter()
        O.mine_batch(od, w.batch.subset(idx), w.settings, 1)
        one_t += time.perf_counter() - t0
        one_pairs += len(idx)
        k1 += 1
    cpu_model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    cpu_model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"value": done_pairs / t_used, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"{done_pairs} random pairs of the same workload ({done_cells} cells), "
                      f"{t_used:.1f} s, OpenMP over pairs",
            "gcups": done_cells * len({g for g, _ in w.settings}) / t_used / 1e9,
            "single_thread": {"value": one_pairs / one_t, "unit": UNIT, "cores": 1,
                              "sample": f"{one_pairs} random pairs, {one_t:.1f} s"},
            "cpu": cpu_model, "nproc": os.cpu_count()}


# --------------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1509_08639_gb300 import synth
    w = synth.workload(args.workload, n_pairs=args.pairs)
    from oracle import oracle as O
    od = O.OracleDict(w.dictionary)
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    S, T = w.batch.sizes()
    sample = max(threads * 8, 64)
    times, pairs = [], []
    for step in range(args.warmup + args.steps):
        idx = rng.choice(w.batch.n_pairs, min(sample, w.batch.n_pairs), replace=False)
        sub = w.batch.subset(idx)
        t0 = time.perf_counter()
        _, used = O.mine_batch(od, sub, w.settings, threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pairs.append(len(idx))
    v = sum(pairs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w.name, "pairs": w.batch.n_pairs},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": int(used), "kind": "oracle",
                             "sample": f"{sample} random pairs per step, OpenMP over pairs"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GB300 arm

def extras_run(ctx, w, dh, reps=3):
    """Bidirectional mining (both dictionaries, union of the selections) and
    the tuning objective (F1 of a 64-setting sweep against the generator's
    planted pairs) on the benchmark batch, each through its host-buffer call:
    wall time per call (inputs copied in, results copied out) and the device
    time of every kernel from one profiled call."""
    from paper_1509_08639_gb300 import mine, synth
    b = w.batch
    P = b.n_pairs
    S, T = b.sizes()
    inv = synth.reverse_dictionary(w.dictionary)
    hb = ctx.dict_create(inv)
    do, so, tk = (np.ascontiguousarray(x, np.int32) for x in (b.doc_off, b.sent_off, b.tokens))
    n = len(w.settings)
    g = np.asarray([s_[0] for s_ in w.settings], np.int32)
    th = np.asarray([s_[1] for s_ in w.settings], np.int32)
    bc = mine.BatchC(P, so.shape[0] - 1, tk.shape[0], mine._ptr(do), mine._ptr(so), mine._ptr(tk))
    sc = mine.SettingsC(n, mine._ptr(g), mine._ptr(th))
    cap = 2 * int(n * np.minimum(S, T).sum())
    outs = (np.zeros(P * n, np.int32), np.zeros(P * n, np.int32), np.zeros(P * n, np.int32),
            np.zeros(P * n + 1, np.int64), np.zeros((cap, 3), np.int32), cap)

    def timed(fn):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        wall = (time.perf_counter() - t0) / reps
        ctx.profile(True)
        ctx.profile_read()
        fn()
        prof = {k: v[0] for k, v in ctx.profile_read().items() if v[1]}
        ctx.profile(False)
        return wall, prof

    wall, prof = timed(lambda: ctx.run_batch_bidi_raw(dh, hb, bc, sc, outs))
    n_union = int(outs[2].sum())
    bidi = {"value": P / wall, "unit": UNIT, "ms_per_call": wall * 1e3,
            "device_ms": sum(prof.values()), "kernel_ms": prof,
            "selected_union": n_union,
            "how": "mine_run_batch_bidi, host buffers, %d calls after 1 warm-up; second dictionary = "
                   "the inverse of the first with 20%% of its entries dropped and one random entry "
                   "added to 30%% of its keys (%d keys)" % (reps, inv.n_keys)}
    sweep = [(gg, tt) for gg in synth.SWEEP_GAPS for tt in synth.SWEEP_THRESHOLDS]
    truth = synth.truth_of(b, w.planted)
    res = {}

    def tune():
        res["r"] = ctx.tune_f1(dh, b, sweep, truth)

    wall_t, prof_t = timed(tune)
    tp, nsel, nt, best = res["r"]
    f1 = 2 * tp[best] / max(nsel[best] + nt, 1)
    tuning = {"value": P / wall_t, "unit": UNIT, "ms_per_call": wall_t * 1e3,
              "device_ms": sum(prof_t.values()), "kernel_ms": prof_t,
              "settings": len(sweep), "distinct_gaps": len(synth.SWEEP_GAPS),
              "best": {"gap": sweep[best][0], "threshold": sweep[best][1], "f1": f1,
                       "tp": tp[best], "selected": nsel[best], "known": nt},
              "how": "mine_tune_f1 over 8 gaps x 8 thresholds against the planted pairs, host "
                     "buffers, %d calls after 1 warm-up" % reps}
    # the contrast without the path constraint: each source sentence's best target
    thr = w.settings[0][1]
    ns = np.zeros(P, np.int32)
    rep = np.zeros(P, np.int32)
    off = np.zeros(P + 1, np.int64)
    bsel = np.zeros((int(so.shape[0] - 1), 3), np.int32)

    def run_best():
        mine._check(ctx.L.mine_best_match(ctx.h, dh, ctypes.byref(bc), int(thr), mine._ptr(ns), mine._ptr(rep),
                                          mine._ptr(off), mine._ptr(bsel), int(bsel.shape[0])), ctx.L)

    wall_b, prof_b = timed(run_best)
    best_match = {"value": P / wall_b, "unit": UNIT, "ms_per_call": wall_b * 1e3,
                  "device_ms": sum(prof_b.values()), "kernel_ms": prof_b, "threshold": thr,
                  "selected": int(ns.sum()), "repeated_targets": int(rep.sum()),
                  "how": "mine_best_match (each source sentence takes its best target; no path "
                         "constraint), host buffers, %d calls after 1 warm-up" % reps}
    ctx.dict_destroy(hb)
    return bidi, tuning, best_match


def config_record(ctx, cfg, reps=5, cpu_budget=8.0):
    """One of the other workloads, measured the same way as the benchmark
    batch: the strategy table tuned on it, the device-resident step (graph
    replay, CUDA events), the host-buffer call end to end (pinned arrays,
    one call at a time), and the oracle on a bounded sample."""
    import torch
    from paper_1509_08639_gb300 import mine, synth
    t_gen = time.perf_counter()
    w = synth.workload(cfg)
    t_gen = time.perf_counter() - t_gen
    b = w.batch
    P = b.n_pairs
    S, T = b.sizes()
    n_set = len(w.settings)
    n_gap = len({g for g, _ in w.settings})
    cells = int((S.astype(np.int64) * T).sum())
    dh = ctx.dict_create(w.dictionary)
    old_tab = ctx.align_strategy()
    t_tune = time.perf_counter()
    table = ctx.autotune_batch(dh, b, w.settings)
    t_tune = time.perf_counter() - t_tune
    dev = torch.device("cuda", torch.cuda.current_device())
    sent = torch.from_numpy(b.sent_off).to(dev)
    tok = torch.from_numpy(b.tokens).to(dev)
    cap = max(int(n_set * np.minimum(S, T).astype(np.int64).sum()), 1)
    nw = torch.zeros(P * n_set, dtype=torch.int32, device=dev)
    ns = torch.zeros(P * n_set, dtype=torch.int32, device=dev)
    sel = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)
    n_sent, n_tok = int(b.sent_off.shape[0] - 1), int(b.tokens.shape[0])

    def step():
        ctx.run_batch_device(dh, P, b.doc_off, sent, tok, n_sent, n_tok, w.settings, nw, ns, sel, cap, stream)

    for _ in range(3):
        step()
    stream.synchronize()
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    ctx.profile(True)
    ctx.profile_read()
    step()
    stream.synchronize()
    prof = {k: v[0] for k, v in ctx.profile_read().items() if v[1]}
    ctx.profile(False)
    # end to end: pinned host arrays through mine_run_batch
    pin_sent = torch.from_numpy(b.sent_off).pin_memory()
    pin_tok = torch.from_numpy(b.tokens).pin_memory()
    hdo = np.ascontiguousarray(b.doc_off)
    g = np.asarray([x[0] for x in w.settings], np.int32)
    th = np.asarray([x[1] for x in w.settings], np.int32)
    bc = mine.BatchC(P, n_sent, n_tok, mine._ptr(hdo), pin_sent.data_ptr(), pin_tok.data_ptr())
    sc = mine.SettingsC(n_set, mine._ptr(g), mine._ptr(th))
    outs = (torch.zeros(P * n_set, dtype=torch.int32).pin_memory().numpy(),
            torch.zeros(P * n_set, dtype=torch.int32).pin_memory().numpy(),
            torch.zeros(P * n_set + 1, dtype=torch.int64).pin_memory().numpy(),
            torch.zeros(cap * 3, dtype=torch.int32).pin_memory().numpy(), cap)
    ctx.run_batch_raw(dh, bc, sc, outs)
    io0 = ctx.io_bytes()
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.run_batch_raw(dh, bc, sc, outs)
    e2e_s = (time.perf_counter() - t0) / reps
    io1 = ctx.io_bytes()
    assert np.array_equal(outs[0], nw.cpu().numpy()) and np.array_equal(outs[1], ns.cpu().numpy())
    cpu = cpu_baseline(w, budget_s=cpu_budget)
    ctx.align_strategy(old_tab)
    ctx.dict_destroy(dh)
    return {"workload": w.name, "pairs": P, "cells": cells, "settings": n_set, "distinct_gaps": n_gap,
            "tokens": n_tok, "ms_per_step": ms, "value": P / (ms / 1e3), "unit": UNIT,
            "gcups": cells * n_gap / (ms / 1e3) / 1e9, "kernel_ms": prof,
            "e2e": {"value": P / e2e_s, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                    "h2d_bytes_per_step": (io1[0] - io0[0]) // reps,
                    "d2h_bytes_per_step": (io1[1] - io0[1]) // reps,
                    "how": "mine_run_batch, pinned host inputs and outputs, one call at a time"},
            "cpu_baseline": cpu, "generation_s": t_gen, "autotune_s": t_tune,
            "autotune": {str(k): v for k, v in enumerate(table) if v >= 0}}


def saturated_alignment(ctx, dh, n_sms, settings, reps=5):
    """The alignment kernel on a load that keeps every warp busy to the end:
    32 pairs per SM of 32 x 1024 sentences (one warp each, no tail), three
    tokens per sentence, through the device-resident call; k_align's time from
    the per-kernel events."""
    import torch
    rng = np.random.default_rng(1519)
    P, S, T, L = 32 * n_sms, 32, 1024, 3
    n_sent = P * (S + T)
    doc = np.zeros(2 * P + 1, np.int32)
    doc[1::2] = S
    doc[2::2] = T
    doc = np.cumsum(doc).astype(np.int32)
    sent = np.arange(n_sent + 1, dtype=np.int32) * L
    tok = rng.integers(0, 20000, n_sent * L).astype(np.int32)
    dev = torch.device("cuda", torch.cuda.current_device())
    sent_d, tok_d = torch.from_numpy(sent).to(dev), torch.from_numpy(tok).to(dev)
    cap = len(settings) * P * S
    nw = torch.zeros(P * len(settings), dtype=torch.int32, device=dev)
    ns = torch.zeros_like(nw)
    sel = torch.zeros(3 * cap, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream(dev)

    def step():
        ctx.run_batch_device(dh, P, doc, sent_d, tok_d, n_sent, int(tok.shape[0]), settings, nw, ns, sel, cap, st)
    for _ in range(3):
        step()
    st.synchronize()
    ctx.check()
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(reps):
        step()
    st.synchronize()
    pr = ctx.profile_read()
    ctx.profile(False)
    ctx.check()
    t = pr["k_align"][0] / reps / 1e3
    cells = P * S * T
    return {"pairs": P, "shape": [S, T], "ms": t * 1e3, "gcups": cells / t / 1e9,
            "achieved": 4 * cells / t / 1e12, "unit": "Tops/s",
            "how": "32 x 1024-sentence pairs, 32 per SM, one warp each (no tail): k_align per launch"}


def serving_run(ctx, dh, rate, seconds):
    """Poisson arrivals of 40x45 pairs with a 1% tail of 2000x2000 pairs."""
    from paper_1509_08639_gb300 import synth
    # a pool of pairs drawn like config 5's (cycled when the run needs more)
    w5 = synth.workload(5, n_pairs=min(max(int(rate * seconds * 1.1) + 16, 64), 4000))
    # the request pool uses its own dictionary: register it
    dh5 = ctx.dict_create(w5.dictionary)
    arrivals = synth.poisson_arrivals(rate, seconds)
    n = len(arrivals)
    docs = [w5.batch.pair(p % w5.batch.n_pairs) for p in range(n)]
    lat = []
    done = threading.Event()
    got = [0]

    def poller():
        while got[0] < n:
            for r in ctx.poll(1024, 20000):
                lat.append(r[5])
                got[0] += 1
        done.set()

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for k in range(n):
        now = time.perf_counter() - t0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        src, tgt = docs[k]
        ctx.submit(dh5, src, tgt, w5.settings)
    done.wait(120)
    t1 = time.perf_counter() - t0
    th.join(5)
    lat = np.asarray(lat, np.float64) / 1e6
    return {"offered_pairs_per_s": rate, "served_pairs_per_s": n / t1, "requests": n,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "workload": "40x45 pairs, 1% 2000x2000, Poisson arrivals"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1509_08639_gb300 import mine, synth

    # every rank mines its own batch (independent pairs: weak scaling)
    w = synth.workload(args.workload, n_pairs=args.pairs, seed=rank_seed(args.workload, rank))
    b = w.batch
    P = b.n_pairs
    S, T = b.sizes()
    n_set = len(w.settings)
    n_gap = len({g for g, _ in w.settings})
    cells = int((S * T).sum())
    ctx = mine.Context(device=local)
    dh = ctx.dict_create(w.dictionary)
    int_peak, int_peak_forms = mine.int_peak(local)
    int_peak_tops = int_peak / 1e12
    # alignment strategy per size bin, timed on this GPU
    t_tune = time.perf_counter()
    align_table = ctx.align_strategy() if args.no_autotune else ctx.autotune_batch(dh, w.batch, w.settings)
    t_tune = time.perf_counter() - t_tune

    # ---- device-resident inputs
    sent = torch.from_numpy(b.sent_off).to(dev)
    tok = torch.from_numpy(b.tokens).to(dev)
    cap = max(int(n_set * np.minimum(S, T).sum()), 1)
    nw = torch.zeros(P * n_set, dtype=torch.int32, device=dev)
    ns = torch.zeros(P * n_set, dtype=torch.int32, device=dev)
    sel = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)
    n_sent, n_tok = int(b.sent_off.shape[0] - 1), int(b.tokens.shape[0])

    def step():
        ctx.run_batch_device(dh, P, b.doc_off, sent, tok, n_sent, n_tok, w.settings,
                             nw, ns, sel, cap, stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    ctx.check()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        clk.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
    barrier()
    launches = ctx.launch_count() - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, ws)
    # per-kernel device times: a separate pass with CUDA events around every
    # launch on the launch stream (plain launches instead of the graph)
    prof_steps = max(1, min(args.steps, 5))
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(prof_steps):
        step()
    stream.synchronize()
    prof = {k: (v[0] / prof_steps, v[1] / prof_steps) for k, v in ctx.profile_read().items()}
    ctx.profile(False)
    if args.only_device:
        if rank == 0:
            print(json.dumps({"workload": w.name, "pairs": P, "ms_per_step": ms,
                              "pairs_per_s": P / (ms / 1e3),
                              "kernel_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]}}),
                  flush=True)
        ctx.close()
        return
    value = whole_job_rate(P, ws, ms / 1e3)
    gcups = ws * cells * n_gap / (ms / 1e3) / 1e9

    # ---- end to end through the host-buffer calls (pinned host memory).
    # Every step copies its inputs in and its results out inside the timed
    # region.  Headline: two calls in flight (mine_run_batch_async, each with
    # its own pinned outputs), so one call's input copies overlap the kernels
    # of the call before it; also timed one call at a time (mine_run_batch).
    pin_sent = torch.from_numpy(b.sent_off).pin_memory()
    pin_tok = torch.from_numpy(b.tokens).pin_memory()
    hdo = np.ascontiguousarray(b.doc_off)
    g = np.asarray([s[0] for s in w.settings], np.int32)
    th = np.asarray([s[1] for s in w.settings], np.int32)
    bc = mine.BatchC(P, n_sent, n_tok, mine._ptr(hdo), pin_sent.data_ptr(), pin_tok.data_ptr())
    sc = mine.SettingsC(n_set, mine._ptr(g), mine._ptr(th))

    def pinned_outs():
        return (torch.zeros(P * n_set, dtype=torch.int32).pin_memory().numpy(),
                torch.zeros(P * n_set, dtype=torch.int32).pin_memory().numpy(),
                torch.zeros(P * n_set + 1, dtype=torch.int64).pin_memory().numpy(),
                torch.zeros(cap * 3, dtype=torch.int32).pin_memory().numpy(), cap)

    outs2 = [pinned_outs(), pinned_outs()]

    def pipelined(k_steps):
        pending = []
        for k in range(k_steps):
            if len(pending) == 2:
                ctx.batch_wait_raw(pending.pop(0))
            pending.append(ctx.run_batch_async_raw(dh, bc, sc, outs2[k % 2]))
        for t in pending:
            ctx.batch_wait_raw(t)

    pipelined(max(args.warmup, 2))
    io0 = ctx.io_bytes()
    barrier()
    t0 = time.perf_counter()
    pipelined(args.steps)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, ws)
    io1 = ctx.io_bytes()
    outs = outs2[0]
    for _ in range(args.warmup):
        ctx.run_batch_raw(dh, bc, sc, outs)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.run_batch_raw(dh, bc, sc, outs)
    e2e_sync_s = max_over_ranks((time.perf_counter() - t0) / args.steps, ws)
    # device-resident results equal the host-call results
    for o in outs2:
        assert np.array_equal(nw.cpu().numpy(), o[0]) and np.array_equal(ns.cpu().numpy(), o[1])

    # ---- plain path: one pair per call
    plain = None
    if args.plain_pairs > 0:
        idx = np.random.default_rng(3).choice(P, min(args.plain_pairs, P), replace=False)
        subs = [b.subset([p]) for p in idx]
        for sb in subs[:5]:
            ctx.run_batch(dh, sb, w.settings)
        t0 = time.perf_counter()
        for sb in subs:
            ctx.run_batch(dh, sb, w.settings)
        dt = time.perf_counter() - t0
        plain = {"value": len(subs) / dt, "unit": UNIT, "pairs": len(subs),
                 "how": "one pair per mine_run_batch call (copy in, 4 kernels, copy out, sync)"}

    serving = None
    if not args.no_serving and rank == 0:
        serving = serving_run(ctx, dh, args.serve_rate, args.serve_seconds)
        rates = [float(r) for r in args.serve_sweep.split(",") if r.strip()]
        serving["sweep"] = [serving_run(ctx, dh, r, args.serve_seconds) for r in rates]
    bidi = tuning = best_match = None
    if not args.no_extras and rank == 0:
        bidi, tuning, best_match = extras_run(ctx, w, dh)
    configs = {}
    if rank == 0 and not args.only_device:
        for c in [int(x) for x in args.configs.split(",") if x.strip()]:
            configs[str(c)] = config_record(ctx, c, cpu_budget=4.0 if args.no_cpu else 8.0)

    # ---- roofline of each stage, in algorithmic units:
    # scoring (translate + set build + score matrix) is bounded by HBM: 4 B per
    # score cell written + 4 B per token read, over all its launches together;
    # the alignment is bounded by int32 add/max issue: 4 ops per DP cell
    # (diagonal add, gap add, two maxima) per distinct gap, against the peak
    # measured on this GPU at the start of the run (mine_int_peak).
    hbm_peak, sm_mhz_max, peak_kind = peaks()
    timed = {k: v for k, v in prof.items() if v[1] > 0}
    per_launch_ms = {k: v[0] / v[1] for k, v in timed.items()}
    src_tok = int((b.sent_off[b.doc_off[1:-1:2]].astype(np.int64) -
                   b.sent_off[b.doc_off[0:-1:2]].astype(np.int64)).sum())
    tgt_tok = n_tok - src_tok
    n_src_rows = int(S.sum())
    kept = kept_entries(w)
    score_bytes = 4 * cells + 4 * (src_tok + tgt_tok)
    prep_bytes = 4 * n_tok + 2 * tgt_tok + 4 * kept + 16 * n_src_rows   # sub-figure of k_pairprep
    align_ops = 4 * cells * n_gap
    stages = {"scoring": ("k_pairprep_wide", "k_pairprep", "k_pairprep_xwide", "k_prep", "k_order",
                          "k_score_wide", "k_score", "k_score_xwide"),
              "alignment": ("k_align", "k_align_tiled")}
    rl = {}
    for st_name, ks in stages.items():
        t = sum(per_launch_ms.get(k, 0.0) for k in ks) / 1e3
        if t <= 0:
            continue
        launched = [k for k in ks if k in per_launch_ms]
        if st_name == "scoring":
            a = score_bytes / t / 1e9
            tp = sum(per_launch_ms.get(k, 0.0) for k in ks[:4]) / 1e3
            rl[st_name] = {"bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                           "frac": a / hbm_peak, "traffic": committed_traffic("scoring"),
                           "algorithmic_bytes": score_bytes, "ms": t * 1e3, "launches": launched,
                           "bytes_rule": "4 B per score cell (S*T) + 4 B per source and target token",
                           "preparation_only": {"achieved": prep_bytes / tp / 1e9 if tp > 0 else None,
                                                "unit": "GB/s", "ms": tp * 1e3,
                                                "algorithmic_bytes": prep_bytes,
                                                "bytes_rule": "4 B per token + 2 B per target id + 4 B per kept entry + 16 B per source row"}}
        else:
            a = align_ops / t / 1e12
            rl[st_name] = {"bound": "alu", "achieved": a, "peak": int_peak_tops, "unit": "Tops/s",
                           "frac": a / int_peak_tops, "traffic": committed_traffic("alignment"),
                           "algorithmic_ops": align_ops, "ms": t * 1e3, "launches": launched,
                           "gcups": cells * n_gap / t / 1e9,
                           "ops_rule": "4 int32 ops per DP cell per distinct gap"}
    if "alignment" in rl and rank == 0 and not args.no_extras:
        sat = saturated_alignment(ctx, dh, torch.cuda.get_device_properties(local).multi_processor_count,
                                  [w.settings[0]])
        sat["frac"] = sat["achieved"] / int_peak_tops
        rl["alignment"]["saturated"] = sat
    dom = max(rl, key=lambda k: rl[k]["ms"]) if rl else None
    roof = dict(rl.get(dom, {}))
    roof["stage"] = dom
    roof["peak_kind"] = ("measured: MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind) if roof.get("bound") == "hbm" \
        else "measured: mine_int_peak on this GPU (%s)" % ", ".join("%.1f" % (v / 1e12) for v in int_peak_forms)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": w.name, "pairs": P, "cells": cells, "settings": n_set,
                   "tokens": n_tok, "l2": "inputs larger than L2 (tokens %d MB, score matrices %d MB)"
                   % (4 * n_tok >> 20, 4 * cells >> 20), "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "gcups": gcups,
        "e2e": {"value": whole_job_rate(P, ws, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": (io1[0] - io0[0]) // args.steps,
                "d2h_bytes_per_step": (io1[1] - io0[1]) // args.steps,
                "ms_per_step": e2e_s * 1e3,
                "how": "mine_run_batch_async, two calls in flight, pinned host inputs and outputs",
                "one_call_at_a_time": {"value": whole_job_rate(P, ws, e2e_sync_s), "unit": UNIT,
                                       "ms_per_step": e2e_sync_s * 1e3, "how": "mine_run_batch"}},
        "plain": plain,
        "batched_vs_plain": (value / ws) / plain["value"] if plain else None,
        "serving": serving,
        "bidirectional": bidi,
        "tuning": tuning,
        "best_match": best_match,
        "configs": configs,
        "roofline": roof,
        "roofline_kernels": rl,
        "kernel_ms_per_step": {k: v[0] for k, v in timed.items()},
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "int_peak": {"value": int_peak_tops, "unit": "Tops/s", "forms": [v / 1e12 for v in int_peak_forms],
                     "how": "mine_int_peak: full grid of independent max(x + g, y) chains, ops written counted"},
        "autotune": {"seconds": t_tune,
                     "table": {str(k): {0: "1 warp", 3: "2 warps", 4: "4 warps", 1: "8 warps",
                                        2: "tiles"}[v] for k, v in enumerate(align_table) if v >= 0},
                     "bin": "ceil(log2(S*T+1)); other bins keep the built-in rule",
                     "how": "mine_autotune_batch on the benchmark batch and settings (strategies timed on its alignments)"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
