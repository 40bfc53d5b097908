"""Host-side logic of the benchmark, on the CPU: the count of kept
translations (the entries the preparation kernel writes, part of its
algorithmic bytes), computed with numpy in bench.py, against a direct loop
over pairs, sentences, distinct tokens and dictionary entries; the clock
sampler's choice of the samples taken during the timed region; the committed
DRAM traffic used only while it describes the kernel source; and the
whole-job rate and per-rank seeds of the multi-GPU run."""
import os
import sys
import time

import numpy as np

from paper_1509_08639_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def kept_by_loop(w):
    b, d = w.batch, w.dictionary
    trans = {int(k): [int(t) for t in d.trans[d.trans_off[i]:d.trans_off[i + 1]]]
             for i, k in enumerate(d.keys)}
    total = 0
    for p in range(b.n_pairs):
        (s_off, s_tok), (_, t_tok) = b.pair(p)
        target = set(int(t) for t in t_tok)
        for i in range(s_off.shape[0] - 1):
            for tok in set(int(t) for t in s_tok[s_off[i]:s_off[i + 1]]):
                total += sum(1 for u in trans.get(tok, []) if u in target)
    return total


def test_kept_entries_match_a_direct_count():
    for cfg, n in ((1, None), (2, 40), (5, 30)):
        w = synth.workload(cfg, n_pairs=n)
        want = kept_by_loop(w)
        assert want > 0
        assert bench.kept_entries(w) == want, w.name


def test_kept_entries_of_edge_batches():
    rng = np.random.default_rng(7)
    d = synth.make_dictionary(rng, 500, 3)
    S = np.array([0, 1, 3, 0, 5])
    T = np.array([4, 0, 3, 0, 6])
    b = synth.make_pairs(rng, synth._zipf_cdf(500), d, S, T, np.full(5, 0.5), 1, 9)
    w = synth.Workload("edges", b, d, [], [], [(-65536, 32768)], np.zeros((0, 3), np.int64))
    assert bench.kept_entries(w) == kept_by_loop(w)
    # a dictionary that translates nothing
    w0 = synth.Workload("empty dictionary", b, synth.dictionary_from_map({}), [], [],
                        [(-65536, 32768)], np.zeros((0, 3), np.int64))
    assert bench.kept_entries(w0) == 0


def _fake_smi(tmp_path, flag, stamp=True):
    fake = tmp_path / "nvidia-smi"
    ts = ("datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]" if stamp else "'n/a'")
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import datetime, os, sys, time\n"
        "while True:\n"
        f"    on = os.path.exists({str(flag)!r})\n"
        "    mhz = 2070 if on else 1000\n"
        "    cap = 'Active' if on else 'Not Active'\n"
        f"    ts = {ts}\n"
        "    print(f'{ts}, 0, {mhz}, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, {cap}', flush=True)\n"
        "    time.sleep(0.02)\n")
    fake.chmod(0o755)


def test_clock_sampler_keeps_the_timed_region(tmp_path, monkeypatch):
    """A stand-in for nvidia-smi prints a timestamped sample every 20 ms:
    1000 MHz outside the timed region, 2070 MHz with the power cap active
    while a file exists; the summary keeps the samples of the region."""
    flag = tmp_path / "loaded"
    _fake_smi(tmp_path, flag)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as clk:
        time.sleep(0.1)
        flag.write_text("1")
        time.sleep(0.05)          # the stand-in sees the new state
        clk.mark_start()
        time.sleep(0.3)
        clk.mark_end()
        time.sleep(0.05)
        flag.unlink()
    s = clk.summary()
    assert s["window"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] >= 5
    # no region marked: every sample counts
    with bench.ClockSampler(0) as clk2:
        time.sleep(0.1)
    s2 = clk2.summary()
    assert s2["window"] == "whole sampler run" and s2["sm_mhz"] == 1000.0 and s2["reasons"] == []


def test_clock_sampler_without_readable_timestamps(tmp_path, monkeypatch):
    flag = tmp_path / "loaded"
    _fake_smi(tmp_path, flag, stamp=False)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as clk:
        clk.mark_start()
        time.sleep(0.1)
        clk.mark_end()
    s = clk.summary()
    assert s["window"] == "whole sampler run" and s["samples"] >= 3 and s["sm_mhz"] == 1000.0


def test_traffic_is_kept_only_while_it_describes_the_kernel_source(tmp_path, monkeypatch):
    # a stand-in tree: the three kernel sources and a committed summary keyed by their hash
    csrc = tmp_path / "paper_1509_08639_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("kernels.cu", "align.cu", "internal.h"):
        (csrc / f).write_text("// " + f + "\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    import json
    summary = {"source_hash": bench.kernel_source_hash(),
               "kernels": {"scoring": {"dram_bytes_per_launch_full_workload": 123},
                           "alignment": {"dram_bytes_per_launch_full_workload": 45}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(summary))
    assert bench.committed_traffic("scoring") == 123
    assert bench.committed_traffic("alignment") == 45
    assert bench.committed_traffic("other") is None
    # any change to a kernel source: the counters no longer describe it
    (csrc / "align.cu").write_text("// align.cu, changed\n")
    assert bench.committed_traffic("scoring") is None
    # no summary at all
    (tmp_path / "profiles" / "traffic.json").unlink()
    assert bench.committed_traffic("scoring") is None


def test_whole_job_rate_and_rank_seeds():
    # units of all ranks over the slowest rank's time
    assert bench.whole_job_rate(10000, 1, 0.002) == 5e6
    assert bench.whole_job_rate(10000, 4, 0.004) == 1e7
    # rank 0 mines the standard batch; other ranks batches of their own, distinct per rank
    assert bench.rank_seed(2, 0) is None
    seeds = {bench.rank_seed(2, r) for r in range(1, 8)}
    assert len(seeds) == 7 and all(s != 1508 + 2 for s in seeds)
    assert bench.max_over_ranks(3.5, 1) == 3.5
