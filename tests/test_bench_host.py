"""Host-side arithmetic of the benchmark's roofline, on the CPU: the count
of kept translations (the entries the preparation kernel writes, part of
its algorithmic bytes), computed with numpy in bench.py, against a direct
loop over pairs, sentences, distinct tokens and dictionary entries."""
import os
import sys

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
