"""Seeded synthetic comparable corpora and bilingual dictionaries.

This module makes INPUTS only. It holds none of the miner's arithmetic (no
scoring, no alignment, no selection), so both the CPU oracle and the CUDA path
may take their inputs from it.

The paper mines 1,000 random Polish-English Wikipedia article pairs (Table 3)
with a classifier trained on real corpora (Table 1). Neither the articles nor
the corpora exist here, so seeded synthetic documents stand in for them:

* token IDs follow a Zipf law, P(rank r) ~ r^-1.1, token ID = rank - 1, over
  one vocabulary per language (Table 1 gives vocabularies of 25k-1.2M words;
  20k and 200k are used);
* the dictionary has one key per source ID with 1..kmax translations; the first
  translation of source rank r is target rank r (frequent maps to frequent),
  the others are distinct and uniform over the target vocabulary;
* a chosen fraction of target sentences are noisy in-order translations of
  source sentences (each source token becomes one of its translations, then a
  5% drop and a 5% insertion of a random Zipf token per token); the others are
  random Zipf sentences.

A batch is packed CSR: ``doc_off[2P+1]`` (sentence ranges; document 2p is the
source article of pair p, 2p+1 its target), ``sent_off[N_sent+1]`` (token
ranges) and ``tokens[N_tok]`` (int32).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Q16_ONE = 65536


def q16(x: float) -> int:
    """Round a real to Q16 (x * 65536), halves away from zero (llround)."""
    y = x * Q16_ONE
    return int(math.floor(y + 0.5)) if y >= 0 else -int(math.floor(-y + 0.5))


@dataclasses.dataclass
class Dictionary:
    """Bilingual dictionary in CSR form: key k -> trans[trans_off[k]:trans_off[k+1]]."""
    keys: np.ndarray        # int32[E], unique, >= 0
    trans_off: np.ndarray   # int32[E+1]
    trans: np.ndarray       # int32[sum k]

    @property
    def n_keys(self) -> int:
        return int(self.keys.shape[0])


@dataclasses.dataclass
class Batch:
    """P article pairs in packed CSR form (see module docstring)."""
    doc_off: np.ndarray     # int32[2P+1]
    sent_off: np.ndarray    # int32[N_sent+1]
    tokens: np.ndarray      # int32[N_tok]

    @property
    def n_pairs(self) -> int:
        return (int(self.doc_off.shape[0]) - 1) // 2

    def sizes(self):
        """(S, T) sentence counts per pair, int64 arrays."""
        d = self.doc_off.astype(np.int64)
        return d[1::2] - d[0:-1:2], d[2::2] - d[1::2]

    def doc(self, d: int):
        """Document d as (sent_off rebased to 0, tokens) numpy views/copies."""
        s0, s1 = int(self.doc_off[d]), int(self.doc_off[d + 1])
        so = self.sent_off[s0:s1 + 1].astype(np.int64)
        t0 = int(so[0])
        return (so - t0).astype(np.int32), self.tokens[t0:int(so[-1])]

    def pair(self, p: int):
        """((src_off, src_tok), (tgt_off, tgt_tok)) of pair p."""
        return self.doc(2 * p), self.doc(2 * p + 1)

    def subset(self, idx) -> "Batch":
        """A new packed batch holding the pairs listed in ``idx`` (in that order)."""
        docs = []
        for p in idx:
            docs.append(self.doc(2 * int(p)))
            docs.append(self.doc(2 * int(p) + 1))
        return pack_docs(docs)


def pack_docs(docs) -> Batch:
    """Pack a list of (sent_off, tokens) documents (src, tgt, src, tgt, ...)."""
    doc_off = [0]
    sent_off = [np.zeros(1, np.int64)]
    toks = []
    ntok = 0
    for so, tk in docs:
        so = np.asarray(so, np.int64)
        doc_off.append(doc_off[-1] + len(so) - 1)
        sent_off.append(so[1:] + ntok)
        ntok += int(so[-1])
        toks.append(np.asarray(tk, np.int32))
    return Batch(np.asarray(doc_off, np.int32),
                 np.concatenate(sent_off).astype(np.int32),
                 np.concatenate(toks).astype(np.int32) if toks else np.zeros(0, np.int32))


def docs_from_lists(sentences_src, sentences_tgt):
    """Pack one pair given as lists of token lists (small hand-made cases)."""
    def one(sents):
        off = np.zeros(len(sents) + 1, np.int64)
        for i, s in enumerate(sents):
            off[i + 1] = off[i] + len(s)
        tk = np.asarray([t for s in sents for t in s], np.int32)
        return off.astype(np.int32), tk
    return pack_docs([one(sentences_src), one(sentences_tgt)])


def dictionary_from_map(m: dict) -> Dictionary:
    """Build a Dictionary from {source_id: [target ids]} (hand-made cases)."""
    keys = sorted(m)
    off = [0]
    tr = []
    for k in keys:
        tr.extend(m[k])
        off.append(len(tr))
    return Dictionary(np.asarray(keys, np.int32), np.asarray(off, np.int32),
                      np.asarray(tr, np.int32))


# --------------------------------------------------------------------------
# random building blocks
# --------------------------------------------------------------------------

def _zipf_cdf(vocab: int, s: float = 1.1) -> np.ndarray:
    w = np.arange(1, vocab + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _zipf(rng, cdf, n) -> np.ndarray:
    u = rng.random(int(n))
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, cdf.shape[0] - 1).astype(np.int32)


def _excl_cumsum(x) -> np.ndarray:
    out = np.zeros(len(x) + 1, np.int64)
    np.cumsum(x, out=out[1:])
    return out


def _seg_gather(pool, starts, lens):
    """Concatenate pool[starts[k]:starts[k]+lens[k]] for all k."""
    lens = np.asarray(lens, np.int64)
    total = int(lens.sum())
    if total == 0:
        return pool[:0].copy()
    off = _excl_cumsum(lens)
    idx = np.arange(total, dtype=np.int64) + np.repeat(np.asarray(starts, np.int64) - off[:-1], lens)
    return pool[idx]


def make_dictionary(rng, vocab: int, kmax: int) -> Dictionary:
    """One key per source ID; k ~ U{1..kmax} translations, first = same rank."""
    k = rng.integers(1, kmax + 1, size=vocab)
    off = _excl_cumsum(k)
    trans = np.empty(int(off[-1]), np.int64)
    trans[off[:-1]] = np.arange(vocab)
    # extra translations: uniform over the target vocabulary, distinct per key
    pos = np.arange(int(off[-1]))
    is_first = np.zeros(int(off[-1]), bool)
    is_first[off[:-1]] = True
    extra_pos = pos[~is_first]
    trans[extra_pos] = rng.integers(0, vocab, size=extra_pos.shape[0])
    # re-draw collisions until every key's list is distinct; among equal
    # entries of one key the first translation sorts first and is kept
    key_of = np.repeat(np.arange(vocab), k)
    for _ in range(64):
        order = np.lexsort((~is_first, trans, key_of))
        sk, st = key_of[order], trans[order]
        dup = np.zeros(st.shape[0], bool)
        dup[1:] = (sk[1:] == sk[:-1]) & (st[1:] == st[:-1])
        bad = order[dup]
        if bad.shape[0] == 0:
            break
        trans[bad] = rng.integers(0, vocab, size=bad.shape[0])
    return Dictionary(np.arange(vocab, dtype=np.int32), off.astype(np.int32),
                      trans.astype(np.int32))


def make_pairs(rng, cdf, d: Dictionary, S, T, frac, len_lo, len_hi,
               p_drop=0.05, p_ins=0.05, planted: list | None = None) -> Batch:
    """P article pairs with S[p] x T[p] sentences; frac[p] of T translated.

    When ``planted`` is a list, an int64 array of (pair, source sentence,
    target sentence) rows, indices local to the pair's articles, is appended
    to it: which target sentence is the translation of which source sentence
    (the random draws are the same either way)."""
    S = np.asarray(S, np.int64)
    T = np.asarray(T, np.int64)
    P = S.shape[0]
    n_tr = np.minimum(np.rint(np.asarray(frac, np.float64) * T).astype(np.int64),
                      np.minimum(S, T))
    nS, nT = int(S.sum()), int(T.sum())
    src_base = _excl_cumsum(S)
    tgt_base = _excl_cumsum(T)

    # source sentences (pool A)
    src_len = rng.integers(len_lo, len_hi + 1, size=nS)
    src_start = _excl_cumsum(src_len)
    src_tok = _zipf(rng, cdf, src_start[-1])

    # which source sentences are translated into which target slots (in order)
    tr_src = np.empty(int(n_tr.sum()), np.int64)
    tr_slot = np.empty(int(n_tr.sum()), np.int64)
    o = 0
    for p in range(P):
        n = int(n_tr[p])
        if n:
            tr_src[o:o + n] = src_base[p] + np.sort(rng.choice(int(S[p]), n, replace=False))
            tr_slot[o:o + n] = tgt_base[p] + np.sort(rng.choice(int(T[p]), n, replace=False))
            o += n
    if planted is not None:
        pair_of_tr = np.repeat(np.arange(P, dtype=np.int64), n_tr)
        planted.append(np.stack([pair_of_tr, tr_src - src_base[pair_of_tr],
                                 tr_slot - tgt_base[pair_of_tr]], axis=1))

    # translated sentences (pool B): dictionary translation, then drop/insert noise
    base = _seg_gather(src_tok, src_start[tr_src], src_len[tr_src]).astype(np.int64)
    cnt = (d.trans_off[1:] - d.trans_off[:-1]).astype(np.int64)
    pick = d.trans_off[base].astype(np.int64) + np.floor(
        rng.random(base.shape[0]) * cnt[base]).astype(np.int64)
    trans_tok = d.trans[pick].astype(np.int32)
    keep = rng.random(base.shape[0]) >= p_drop
    ins = rng.random(base.shape[0]) < p_ins
    ins_tok = _zipf(rng, cdf, base.shape[0])
    inter_tok = np.stack([trans_tok, ins_tok], axis=1).ravel()
    inter_msk = np.stack([keep, ins], axis=1).ravel()
    tr_pool = inter_tok[inter_msk]
    per_tok = keep.astype(np.int64) + ins.astype(np.int64)
    seg = _excl_cumsum(src_len[tr_src])
    cs = _excl_cumsum(per_tok)
    tr_len = cs[seg[1:]] - cs[seg[:-1]]
    tr_start = _excl_cumsum(tr_len)

    # random target sentences (pool C)
    is_tr = np.zeros(nT, bool)
    is_tr[tr_slot] = True
    n_rnd = nT - tr_slot.shape[0]
    rnd_len = rng.integers(len_lo, len_hi + 1, size=n_rnd)
    rnd_start = _excl_cumsum(rnd_len)
    rnd_pool = _zipf(rng, cdf, rnd_start[-1])

    # target slot -> (start, len) in the combined pool [A | B | C]
    offB = int(src_start[-1])
    offC = offB + int(tr_start[-1])
    tgt_start = np.empty(nT, np.int64)
    tgt_len = np.empty(nT, np.int64)
    tgt_start[tr_slot] = offB + tr_start[:-1]
    tgt_len[tr_slot] = tr_len
    rnd_slots = np.nonzero(~is_tr)[0]
    tgt_start[rnd_slots] = offC + rnd_start[:-1]
    tgt_len[rnd_slots] = rnd_len
    pool = np.concatenate([src_tok, tr_pool, rnd_pool]).astype(np.int32)

    # final order: src0, tgt0, src1, tgt1, ...
    doc_len = np.stack([S, T], axis=1).ravel()
    doc_off = _excl_cumsum(doc_len)
    n_sent = int(doc_off[-1])
    doc_of = np.repeat(np.arange(2 * P), doc_len)
    local = np.arange(n_sent) - doc_off[doc_of]
    pair_of = doc_of // 2
    is_src = (doc_of % 2) == 0
    st = np.where(is_src, 0, 0).astype(np.int64)
    ln = np.empty(n_sent, np.int64)
    si = src_base[pair_of] + local
    ti = tgt_base[pair_of] + local
    st[is_src] = src_start[si[is_src]]
    ln[is_src] = src_len[si[is_src]]
    st[~is_src] = tgt_start[ti[~is_src]]
    ln[~is_src] = tgt_len[ti[~is_src]]
    tokens = _seg_gather(pool, st, ln)
    sent_off = _excl_cumsum(ln)
    return Batch(doc_off.astype(np.int32), sent_off.astype(np.int32), tokens.astype(np.int32))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    batch: Batch
    dictionary: Dictionary
    gaps: list          # Q16, <= 0
    thresholds: list    # Q16, in [0, 65536]
    settings: list      # [(gap, threshold)] evaluated for every pair
    planted: np.ndarray = None   # (pair, src, tgt) rows: translated sentences, local indices


WORKLOAD_NAMES = {
    1: "plain-40x45",
    2: "batched-10k-lognormal",
    3: "long-16x4000x4000",
    4: "sweep-100k-powerlaw-64",
    5: "serving-poisson-1pct-2000",
}

SWEEP_GAPS = [-16384 * k for k in range(1, 9)]
SWEEP_THRESHOLDS = [q16(x) for x in np.linspace(0.3, 0.8, 8)]


def _powerlaw_sizes(rng, n, alpha=1.5, lo=2, hi=2000):
    v = np.arange(lo, hi + 1, dtype=np.float64)
    c = np.cumsum(v ** (-alpha))
    c /= c[-1]
    return lo + np.minimum(np.searchsorted(c, rng.random(n), side="right"), hi - lo)


def workload(cfg: int, n_pairs: int | None = None, seed: int | None = None) -> Workload:
    """Build workload ``cfg`` (1..5). ``n_pairs`` truncates the pair count
    (the first n pairs of the same seeded stream are NOT guaranteed to equal a
    prefix of the full batch; use ``Batch.subset`` for exact prefixes)."""
    seed = (1508 + cfg) if seed is None else seed
    rng = np.random.default_rng(seed)
    g1, t1 = -Q16_ONE, Q16_ONE // 2
    if cfg == 1:
        V, kmax, lo, hi = 20000, 3, 5, 30
        d = make_dictionary(rng, V, kmax)
        P = 1 if n_pairs is None else n_pairs
        S = np.full(P, 40)
        T = np.full(P, 45)
        frac = np.full(P, 0.6)
        gaps, thrs = [g1], [t1]
    elif cfg == 2:
        V, kmax, lo, hi = 200000, 4, 5, 40
        d = make_dictionary(rng, V, kmax)
        P = 10000 if n_pairs is None else n_pairs
        S = np.clip(np.rint(rng.lognormal(math.log(60), 1.0, P)), 5, 800).astype(np.int64)
        T = np.clip(np.rint(rng.lognormal(math.log(60), 1.0, P)), 5, 800).astype(np.int64)
        frac = rng.uniform(0.1, 0.7, P)
        gaps, thrs = [g1], [t1]
    elif cfg == 3:
        V, kmax, lo, hi = 20000, 3, 5, 30
        d = make_dictionary(rng, V, kmax)
        P = 16 if n_pairs is None else n_pairs
        S = np.full(P, 4000)
        T = np.full(P, 4000)
        frac = np.full(P, 0.6)
        gaps, thrs = [g1], [t1]
    elif cfg == 4:
        V, kmax, lo, hi = 200000, 4, 5, 40
        d = make_dictionary(rng, V, kmax)
        P = 100000 if n_pairs is None else n_pairs
        S = _powerlaw_sizes(rng, P)
        T = _powerlaw_sizes(rng, P)
        frac = rng.uniform(0.1, 0.7, P)
        gaps, thrs = list(SWEEP_GAPS), list(SWEEP_THRESHOLDS)
    elif cfg == 5:
        V, kmax, lo, hi = 200000, 4, 5, 30
        d = make_dictionary(rng, V, kmax)
        P = 2000 if n_pairs is None else n_pairs
        big = rng.random(P) < 0.01
        S = np.where(big, 2000, 40)
        T = np.where(big, 2000, 45)
        frac = np.full(P, 0.6)
        gaps, thrs = [g1], [t1]
    else:
        raise ValueError(f"unknown workload {cfg}")
    cdf = _zipf_cdf(V)
    planted = []
    b = make_pairs(rng, cdf, d, S, T, frac, lo, hi, planted=planted)
    settings = [(g, t) for g in gaps for t in thrs]
    return Workload(WORKLOAD_NAMES[cfg], b, d, gaps, thrs, settings, planted[0])


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = 1513) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    n = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    return t[t < duration_s]


def random_matrix(rng, S, T, lo=-65536, hi=65536, values=None) -> np.ndarray:
    """An S x T int32 matrix, uniform in [lo, hi] or drawn from ``values``."""
    if values is not None:
        return np.asarray(rng.choice(np.asarray(values, np.int64), size=(S, T)), np.int32)
    return rng.integers(lo, hi + 1, size=(S, T)).astype(np.int32)


# --------------------------------------------------------------------------
# inputs of bidirectional mining and of the tuning objective
# --------------------------------------------------------------------------

def invert_dictionary(d: Dictionary) -> Dictionary:
    """The reverse dictionary (target language -> source language): key t
    lists, in increasing order, every source ID that has t among its
    translations; keys are the target IDs that occur.  Raises if a key would
    get more than 32 translations (the miner's limit per key)."""
    cnt = (d.trans_off[1:] - d.trans_off[:-1]).astype(np.int64)
    src = np.repeat(d.keys.astype(np.int64), cnt)
    tgt = d.trans.astype(np.int64)
    order = np.lexsort((src, tgt))
    tgt, src = tgt[order], src[order]
    if tgt.shape[0]:
        keep = np.ones(tgt.shape[0], bool)
        keep[1:] = (tgt[1:] != tgt[:-1]) | (src[1:] != src[:-1])
        tgt, src = tgt[keep], src[keep]
    keys, first, per = np.unique(tgt, return_index=True, return_counts=True)
    if per.shape[0] and int(per.max()) > 32:
        raise ValueError("a target ID has more than 32 source translations")
    off = np.zeros(keys.shape[0] + 1, np.int64)
    np.cumsum(per, out=off[1:])
    return Dictionary(keys.astype(np.int32), off.astype(np.int32), src.astype(np.int32))


def reverse_dictionary(d: Dictionary, seed: int = 1519, p_drop: float = 0.2,
                       p_add: float = 0.3) -> Dictionary:
    """A target -> source dictionary of its own, standing in for a model
    trained in the other direction: the inverse of ``d`` with each entry
    dropped with probability p_drop and, per key with probability p_add, one
    uniformly drawn source ID added (distinct per key, at most 32).  With the
    exact inverse the score of a pair is the same in both directions (the two
    coverage terms exchange roles), so mining the other way would find
    nothing new."""
    inv = invert_dictionary(d)
    rng = np.random.default_rng(seed)
    cnt = (inv.trans_off[1:] - inv.trans_off[:-1]).astype(np.int64)
    key_of = np.repeat(np.arange(inv.n_keys, dtype=np.int64), cnt)
    keep = rng.random(inv.trans.shape[0]) >= p_drop
    src_vocab = int(d.keys.max()) + 1 if d.n_keys else 1
    add = rng.random(inv.n_keys) < p_add
    add_key = np.nonzero(add)[0].astype(np.int64)
    add_val = rng.integers(0, src_vocab, size=add_key.shape[0])
    k_all = np.concatenate([key_of[keep], add_key])
    v_all = np.concatenate([inv.trans[keep].astype(np.int64), add_val])
    order = np.lexsort((v_all, k_all))
    k_all, v_all = k_all[order], v_all[order]
    if k_all.shape[0]:
        uniq = np.ones(k_all.shape[0], bool)
        uniq[1:] = (k_all[1:] != k_all[:-1]) | (v_all[1:] != v_all[:-1])
        k_all, v_all = k_all[uniq], v_all[uniq]
    per = np.bincount(k_all, minlength=inv.n_keys)
    if per.shape[0] and int(per.max()) > 32:
        raise ValueError("a key would get more than 32 translations")
    off = np.zeros(inv.n_keys + 1, np.int64)
    np.cumsum(per, out=off[1:])
    return Dictionary(inv.keys.copy(), off.astype(np.int32), v_all.astype(np.int32))


def truth_of(batch: Batch, planted) -> np.ndarray:
    """int32[n_sent]: for source sentence k of pair p (global index
    doc_off[2p] + k) the planted target sentence (index in pair p's target
    article), -1 elsewhere (untranslated source sentences and every target
    sentence)."""
    n_sent = int(batch.doc_off[-1])
    truth = np.full(n_sent, -1, np.int32)
    pl = np.asarray(planted, np.int64).reshape(-1, 3)
    if pl.shape[0]:
        truth[batch.doc_off[2 * pl[:, 0]].astype(np.int64) + pl[:, 1]] = pl[:, 2].astype(np.int32)
    return truth
