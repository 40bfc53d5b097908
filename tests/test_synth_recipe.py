"""The synthetic inputs follow their stated recipe (the five workloads of the
benchmark and the parity tests), on the CPU: pair sizes and their
distributions, sentence lengths, vocabularies, the dictionary's shape, the
planted translations (in order, noisy dictionary translations of their source
sentences) and the settings sweep.  Large configurations are checked on a
truncated number of pairs drawn the same way."""
import math

import numpy as np

from paper_1509_08639_gb300 import synth


def sentence_lengths(b):
    return np.diff(b.sent_off.astype(np.int64))


def side_lengths(b, side):
    """Lengths of the source (side 0) or target (side 1) sentences."""
    d = b.doc_off.astype(np.int64)
    out = []
    for p in range(b.n_pairs):
        s0, s1 = d[2 * p + side], d[2 * p + side + 1]
        out.append(np.diff(b.sent_off[s0:s1 + 1].astype(np.int64)))
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def check_dictionary(d, vocab, kmax):
    keys = d.keys.astype(np.int64)
    assert keys.shape[0] == vocab and np.all(keys == np.arange(vocab))
    cnt = np.diff(d.trans_off.astype(np.int64))
    assert cnt.min() >= 1 and cnt.max() <= kmax
    # every count appears, roughly uniformly
    hist = np.bincount(cnt, minlength=kmax + 1)[1:]
    assert np.all(np.abs(hist / vocab - 1.0 / kmax) < 0.02)
    # the first translation is the key's own rank; translations of a key are distinct
    first = d.trans[d.trans_off[:-1]]
    assert np.all(first == keys)
    key_of = np.repeat(keys, cnt)
    pairs = key_of * vocab + d.trans.astype(np.int64)
    assert np.unique(pairs).shape[0] == pairs.shape[0]
    assert d.trans.min() >= 0 and d.trans.max() < vocab


def check_planted(w, frac_lo, frac_hi, sample=200):
    b, d = w.batch, w.dictionary
    S, T = b.sizes()
    pl = w.planted
    # per pair: round(frac T) rows, at most min(S, T), in increasing order on both sides
    counts = np.bincount(pl[:, 0], minlength=b.n_pairs)
    assert np.all(counts <= np.minimum(S, T))
    full = np.minimum(S, T) > np.rint(frac_hi * T)
    ratio = counts[full] / T[full]
    assert ratio.min() >= frac_lo - 0.5 / T[full].min() - 1e-9
    assert ratio.max() <= frac_hi + 0.5 / T[full].min() + 1e-9
    for p in np.unique(pl[:, 0])[:50]:
        rows = pl[pl[:, 0] == p]
        assert np.all(np.diff(rows[:, 1]) > 0) and np.all(np.diff(rows[:, 2]) > 0)
    # a planted target sentence is a noisy translation of its source sentence:
    # most of its tokens are dictionary translations of the source's tokens
    trans = {}
    rng = np.random.default_rng(5)
    hits = total = 0
    for r in pl[rng.choice(pl.shape[0], min(sample, pl.shape[0]), replace=False)]:
        (so, stok), (to, ttok) = b.pair(int(r[0]))
        src = stok[so[r[1]]:so[r[1] + 1]]
        tgt = ttok[to[r[2]]:to[r[2] + 1]]
        allowed = set()
        for t in src:
            t = int(t)
            if t not in trans:
                trans[t] = set(int(x) for x in d.trans[d.trans_off[t]:d.trans_off[t + 1]])
            allowed |= trans[t]
        hits += sum(1 for t in tgt if int(t) in allowed)
        total += len(tgt)
        # 5% drops and 5% insertions around the source's length
        assert abs(len(tgt) - len(src)) <= max(4, len(src) // 2)
    assert hits / total > 0.9


def check_zipf(tokens, vocab):
    assert tokens.min() >= 0 and tokens.max() < vocab
    c = np.bincount(tokens, minlength=vocab)
    # s = 1.1: rank 1 about 2^1.1 times as frequent as rank 2, 10^1.1 as rank 10
    assert 1.6 < c[0] / max(c[1], 1) < 2.8
    assert 8.0 < c[0] / max(c[9], 1) < 18.0


def test_plain_pair():
    w = synth.workload(1)
    b = w.batch
    S, T = b.sizes()
    assert b.n_pairs == 1 and S[0] == 40 and T[0] == 45
    src = side_lengths(b, 0)
    assert src.min() >= 5 and src.max() <= 30
    check_dictionary(w.dictionary, 20000, 3)
    assert w.settings == [(-65536, 32768)]
    assert w.planted.shape[0] == round(0.6 * 45)
    check_planted(w, 0.6, 0.6)


def test_lognormal_batch():
    w = synth.workload(2, n_pairs=3000)
    b = w.batch
    S, T = b.sizes()
    for x in (S, T):
        assert x.min() >= 5 and x.max() <= 800
        assert 52 <= np.median(x) <= 68                       # lognormal median 60
        # sigma 1 in log space: a quarter of the articles below 60 e^-0.674 = 30.5
        assert 0.2 < np.mean(x < 30.5) < 0.3
    src = side_lengths(b, 0)
    assert src.min() >= 5 and src.max() <= 40
    assert abs(src.mean() - 22.5) < 0.5
    check_dictionary(w.dictionary, 200000, 4)
    check_zipf(b.tokens, 200000)
    assert w.settings == [(-65536, 32768)]
    check_planted(w, 0.1, 0.7)


def test_long_pairs():
    w = synth.workload(3, n_pairs=2)
    S, T = w.batch.sizes()
    assert np.all(S == 4000) and np.all(T == 4000)
    src = side_lengths(w.batch, 0)
    assert src.min() >= 5 and src.max() <= 30
    check_planted(w, 0.6, 0.6, sample=50)


def test_powerlaw_sweep():
    w = synth.workload(4, n_pairs=3000)
    S, T = w.batch.sizes()
    v = np.arange(2, 2001, dtype=np.float64)
    pdf = v ** -1.5
    pdf /= pdf.sum()
    for x in (S, T):
        assert x.min() >= 2 and x.max() <= 2000
        for k in (2, 3, 10):
            want = pdf[:k - 1].sum()                            # P(size <= k)
            got = np.mean(x <= k)
            assert abs(got - want) < 4 * math.sqrt(want * (1 - want) / x.shape[0]) + 1e-3
    assert w.gaps == [-16384 * k for k in range(1, 9)]
    assert w.thresholds == [synth.q16(t) for t in np.linspace(0.3, 0.8, 8)]
    assert w.settings == [(g, t) for g in w.gaps for t in w.thresholds]
    assert len(w.settings) == 64
    check_planted(w, 0.1, 0.7)


def test_served_sizes():
    w = synth.workload(5, n_pairs=3000)
    S, T = w.batch.sizes()
    big = S == 2000
    assert np.all(T[big] == 2000) and np.all(S[~big] == 40) and np.all(T[~big] == 45)
    assert 0.003 < big.mean() < 0.02                           # a 1% tail
    src = side_lengths(w.batch, 0)
    assert src.min() >= 5 and src.max() <= 30


def test_poisson_arrivals():
    t = synth.poisson_arrivals(5000.0, 2.0)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] <= 2.0
    assert abs(t.shape[0] - 10000) < 4 * math.sqrt(10000)
    gaps = np.diff(t)
    assert abs(gaps.mean() * 5000.0 - 1.0) < 0.05             # exponential, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05
