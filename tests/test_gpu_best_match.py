"""The contrast without the path constraint (Section 4: an alignment that may
go upward or leftward comes back to sentences already matched; in the limit
every source sentence takes its best target): CUDA path vs CPU oracle,
bit-exact, on lognormal pairs, tile-edge sizes, ties and empty articles.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import mine, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = mine.Context(device=0)
    yield c
    c.close()


def _same(got, want, what):
    assert len(got) == len(want), what
    bad = [p for p in range(len(got)) if got[p] != want[p]]
    assert not bad, f"{what}: {len(bad)} pairs differ, first {bad[:8]}: got {got[bad[0]]!r:.300} want {want[bad[0]]!r:.300}"


def test_best_match_lognormal_batch(ctx):
    w = synth.workload(2, n_pairs=300)
    dh = ctx.dict_create(w.dictionary)
    od = O.OracleDict(w.dictionary)
    for thr in (32768, 0, 65536):
        _same(ctx.best_match(dh, w.batch, thr), O.best_match_batch(od, w.batch, thr), f"theta {thr}")
    # every source sentence the monotone alignment keeps is kept here too
    got = ctx.best_match(dh, w.batch, 32768)
    nw = ctx.run_batch(dh, w.batch, [(-65536, 32768)])
    for p in range(w.batch.n_pairs):
        assert {i for i, _, _ in nw[p][0][1]} <= {i for i, _, _ in got[p][0]}
    assert sum(r for _, r in got) > 0   # repeated targets occur


def test_best_match_edges_and_ties(ctx):
    rng = np.random.default_rng(91)
    d = synth.make_dictionary(rng, 5000, 3)
    cdf = synth._zipf_cdf(5000)
    edges = [0, 1, 31, 32, 33, 65, 129]
    sizes = [(s, t) for s in edges for t in edges]
    S = np.array([s for s, _ in sizes])
    T = np.array([t for _, t in sizes])
    b = synth.make_pairs(rng, cdf, d, S, T, np.full(len(sizes), 0.6), 5, 30)
    # pairs whose target article repeats one sentence: equal scores in a row
    docs = []
    both = [k for k, (s, t) in enumerate(sizes) if s > 0 and t > 0]
    for p, k in enumerate(both[10:14]):
        src = b.doc(2 * k)
        so, tk = b.doc(2 * k + 1)
        one = tk[so[0]:so[1]]
        n = 40 + 7 * p
        docs += [src, (np.arange(n + 1, dtype=np.int32) * len(one), np.tile(one, n))]
    ties = synth.pack_docs(docs)
    dh = ctx.dict_create(d)
    od = O.OracleDict(d)
    for bb, what in ((b, "edges"), (ties, "ties")):
        for thr in (0, 20000):
            _same(ctx.best_match(dh, bb, thr), O.best_match_batch(od, bb, thr), f"{what}, theta {thr}")
