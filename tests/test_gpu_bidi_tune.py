"""Bidirectional mining and the tuning objective: CUDA path vs CPU oracle,
bit-exact.

Section 6 (Table 2, "BI") mines each article pair with classifiers trained in
both directions and keeps what either finds; Section 4 tunes Threshold and
Penalty (Table 2, "NWT").  Here: mine_run_batch_bidi against the oracle's
union of the two directions, and mine_tune_f1 against the oracle's F1 counts
over a sweep of settings.  Sizes span several score tiles and ragged tails;
the full 10,000-pair batch is run and sampled.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import mine, synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = mine.Context(device=0)
    yield c
    c.close()


def bidi_oracle(d_fwd, d_bwd, batch, settings):
    return O.mine_batch_bidi(O.OracleDict(d_fwd), O.OracleDict(d_bwd), batch, settings, THREADS)


def assert_same(got, want, what):
    assert len(got) == len(want), what
    bad = [p for p in range(len(got)) if got[p] != want[p]]
    assert not bad, f"{what}: {len(bad)} pairs differ, first {bad[:8]}: got {got[bad[0]]!r:.300} want {want[bad[0]]!r:.300}"


def _edge_batch(rng, d, sizes, vocab, lo=5, hi=30):
    cdf = synth._zipf_cdf(vocab)
    S = np.array([s for s, _ in sizes])
    T = np.array([t for _, t in sizes])
    return synth.make_pairs(rng, cdf, d, S, T, np.full(len(sizes), 0.6), lo, hi)


def test_bidi_hand_examples(ctx):
    g = json.load(open(os.path.join(GOLD, "bidi_hand_examples.json")))
    for c in g["cases"]:
        df = synth.dictionary_from_map({int(k): v for k, v in c["fwd_dictionary"].items()})
        db = synth.dictionary_from_map({int(k): v for k, v in c["bwd_dictionary"].items()})
        b = synth.docs_from_lists(c["src"], c["tgt"])
        hf, hb = ctx.dict_create(df), ctx.dict_create(db)
        got = ctx.run_batch_bidi(hf, hb, b, [(g["gap"], g["theta"])])
        assert got[0][0] == (c["nw_fwd"], c["nw_bwd"], [tuple(t) for t in c["union"]]), c["name"]
        ctx.dict_destroy(hf)
        ctx.dict_destroy(hb)


def test_bidi_lognormal_batch(ctx):
    w = synth.workload(2, n_pairs=300)
    inv = synth.reverse_dictionary(w.dictionary)
    hf, hb = ctx.dict_create(w.dictionary), ctx.dict_create(inv)
    settings = w.settings + [(-16384, 16384), (-131072, 49152), (0, 65536)]
    got = ctx.run_batch_bidi(hf, hb, w.batch, settings)
    want = bidi_oracle(w.dictionary, inv, w.batch, settings)
    assert_same(got, want, "bidirectional, 300 lognormal pairs")
    # the backward direction finds pairs the forward one misses
    extra = sum(len(got[p][0][2]) for p in range(len(got)))
    fwd = ctx.run_batch(hf, w.batch, w.settings)
    assert extra > sum(len(fwd[p][0][1]) for p in range(len(fwd)))


def test_bidi_edges(ctx):
    rng = np.random.default_rng(81)
    d = synth.make_dictionary(rng, 5000, 3)
    inv = synth.reverse_dictionary(d, seed=81)
    edges = [0, 1, 2, 31, 32, 33, 63, 64, 65, 129]
    sizes = [(s, t) for s in edges for t in edges] + [(300, 600), (520, 40)]
    b = _edge_batch(rng, d, sizes, 5000)
    settings = [(-65536, 32768), (-20000, 0), (0, 65536)]
    hf, hb = ctx.dict_create(d), ctx.dict_create(inv)
    assert_same(ctx.run_batch_bidi(hf, hb, b, settings), bidi_oracle(d, inv, b, settings), "bidi edges")
    # a reverse dictionary that translates nothing: the union is the forward selection
    empty = synth.dictionary_from_map({})
    he = ctx.dict_create(empty)
    got = ctx.run_batch_bidi(hf, he, b, settings[:1])
    fwd = ctx.run_batch(hf, b, settings[:1])
    assert [[r[0][2]] for r in got] == [[r[0][1]] for r in fwd]
    # the same dictionary both ways round on identical articles
    docs = []
    for p in range(6):
        docs += [b.doc(2 * p + 40), b.doc(2 * p + 40)]
    same = synth.pack_docs(docs)
    hs = ctx.dict_create(synth.dictionary_from_map({k: [k] for k in range(5000)}))
    assert_same(ctx.run_batch_bidi(hs, hs, same, settings),
                bidi_oracle(synth.dictionary_from_map({k: [k] for k in range(5000)}),
                            synth.dictionary_from_map({k: [k] for k in range(5000)}), same, settings),
                "identical articles")


def test_bidi_full_size_batch(ctx):
    """All 10,000 pairs mined both ways against the oracle's union."""
    w = synth.workload(2)
    inv = synth.reverse_dictionary(w.dictionary)
    hf, hb = ctx.dict_create(w.dictionary), ctx.dict_create(inv)
    got = ctx.run_batch_bidi(hf, hb, w.batch, w.settings)
    want = bidi_oracle(w.dictionary, inv, w.batch, w.settings)
    assert_same(got, want, "bidirectional, 10,000 pairs")


def test_bidi_exact_inverse_scores_both_ways_alike(ctx):
    """With the exact inverse dictionary the backward score matrix is the
    transpose of the forward one, so both alignments reach the same optimum."""
    w = synth.workload(2, n_pairs=200)
    inv = synth.invert_dictionary(w.dictionary)
    hf, hb = ctx.dict_create(w.dictionary), ctx.dict_create(inv)
    got = ctx.run_batch_bidi(hf, hb, w.batch, w.settings + [(-16384, 16384)])
    assert all(r[0] == r[1] for row in got for r in row)
    assert_same(got, bidi_oracle(w.dictionary, inv, w.batch, w.settings + [(-16384, 16384)]),
                "exact inverse")


def _f1_oracle(d, batch, settings, truth):
    res, _ = O.mine_batch(O.OracleDict(d), batch, settings, THREADS)
    tp, nsel, nt = O.f1_counts(res, batch, truth)
    return tp, nsel, nt, O.best_setting(tp, nsel, nt)


def test_tune_f1_sweep_64_settings(ctx):
    w = synth.workload(2, n_pairs=300)
    settings = [(g, t) for g in synth.SWEEP_GAPS for t in synth.SWEEP_THRESHOLDS]
    truth = synth.truth_of(w.batch, w.planted)
    dh = ctx.dict_create(w.dictionary)
    got = ctx.tune_f1(dh, w.batch, settings, truth)
    want = _f1_oracle(w.dictionary, w.batch, settings, truth)
    assert got == want
    assert got[2] == w.planted.shape[0] and max(got[0]) > 0


def test_tune_f1_edges(ctx):
    rng = np.random.default_rng(82)
    d = synth.make_dictionary(rng, 5000, 3)
    sizes = [(0, 5), (5, 0), (1, 1), (33, 65), (64, 31), (129, 129)]
    planted = []
    cdf = synth._zipf_cdf(5000)
    S = np.array([s for s, _ in sizes])
    T = np.array([t for _, t in sizes])
    b = synth.make_pairs(rng, cdf, d, S, T, np.full(len(sizes), 0.6), 5, 30, planted=planted)
    truth = synth.truth_of(b, planted[0])
    # entries of target sentences are ignored whatever they hold
    do = b.doc_off
    for p in range(b.n_pairs):
        truth[int(do[2 * p + 1]):int(do[2 * p + 2])] = 0
    settings = [(-65536, 32768), (-20000, 0), (0, 65536), (-65536, 32768)]
    dh = ctx.dict_create(d)
    got = ctx.tune_f1(dh, b, settings, truth)
    assert got == _f1_oracle(d, b, settings, truth)
    assert got[3] != 3   # settings 0 and 3 are equal: the lower index wins
    # nothing known
    none = np.full(truth.shape[0], -1, np.int32)
    got = ctx.tune_f1(dh, b, settings, none)
    assert got == _f1_oracle(d, b, settings, none) and got[2] == 0 and got[0] == [0] * 4
    # a known pair outside its target article is refused
    bad = truth.copy()
    bad[int(do[6])] = int(T[3])
    with pytest.raises(mine.MineError):
        ctx.tune_f1(dh, b, settings, bad)
