"""CUDA path vs CPU oracle, bit-exact (every value is an integer).

All calls go through the C ABI (libmine.so).  Sizes span several tiles (32
source rows x 32 target columns per score tile, 32-row alignment stripes,
16-column direction words) and ragged tails; the full-size batch of 10,000
lognormal pairs is run in the benchmark's launch configuration and sampled.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import mine, synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def ctx():
    c = mine.Context(device=0)
    yield c
    c.close()


def oracle_results(w, batch=None, settings=None):
    res, _ = O.mine_batch(O.OracleDict(w.dictionary), batch or w.batch,
                          settings or w.settings, THREADS)
    return res


def assert_same(got, want, what):
    assert len(got) == len(want), what
    bad = [p for p in range(len(got)) if got[p] != want[p]]
    assert not bad, f"{what}: {len(bad)} pairs differ, first {bad[:8]}: got {got[bad[0]]!r:.300} want {want[bad[0]]!r:.300}"


def test_plain_40x45_pair(ctx):
    w = synth.workload(1)
    dh = ctx.dict_create(w.dictionary)
    got = ctx.run_batch(dh, w.batch, w.settings)
    assert_same(got, oracle_results(w), w.name)
    assert len(got[0][0][1]) > 0


def test_lognormal_batch_subset(ctx):
    w = synth.workload(2, n_pairs=300)
    dh = ctx.dict_create(w.dictionary)
    got = ctx.run_batch(dh, w.batch, w.settings)
    assert_same(got, oracle_results(w), w.name)


def test_full_size_lognormal_batch(ctx):
    """The 10,000-pair batch through the device entry point, as bench.py runs
    it: every pair against the oracle (about 25 s on 16 host cores)."""
    torch = pytest.importorskip("torch")
    w = synth.workload(2)
    b = w.batch
    dh = ctx.dict_create(w.dictionary)
    dev = torch.device("cuda:0")
    sent = torch.from_numpy(b.sent_off).to(dev)
    tok = torch.from_numpy(b.tokens).to(dev)
    P, n = b.n_pairs, len(w.settings)
    S, T = b.sizes()
    cap = int(n * np.minimum(S, T).sum())
    nw = torch.zeros(P * n, dtype=torch.int32, device=dev)
    ns = torch.zeros(P * n, dtype=torch.int32, device=dev)
    sel = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # twice: the second call replays the captured graph
    for _ in range(2):
        ctx.run_batch_device(dh, P, b.doc_off, sent, tok, int(b.sent_off.shape[0] - 1),
                             int(b.tokens.shape[0]), w.settings, nw, ns, sel, cap, stream)
    torch.cuda.synchronize()
    ctx.check()
    nw, ns, sel = nw.cpu().numpy(), ns.cpu().numpy(), sel.cpu().numpy().reshape(-1, 3)
    base = np.zeros(P + 1, np.int64)
    np.cumsum(n * np.minimum(S, T), out=base[1:])
    got = [[(int(nw[p]), [tuple(int(v) for v in t) for t in sel[base[p]:base[p] + ns[p]]])]
           for p in range(P)]
    assert_same(got, oracle_results(w), "10,000 lognormal pairs")
    assert int(ns.sum()) > 0


def test_q16_score_matrices_cell_by_cell(ctx):
    """Every cell of the fixed-point score matrix M against the oracle's: 300
    lognormal pairs, tile-edge sizes, empty sentences, sentences of up to 1024
    tokens, a target article of 8,192-16,384 distinct tokens (the extra-wide
    launches), one with more (the token-keyed path) and a short one with
    4,097-6,144."""
    rng = np.random.default_rng(316)
    w = synth.workload(2, n_pairs=300)
    d = w.dictionary
    edges = [0, 1, 2, 31, 32, 33, 63, 64, 65, 129]
    edge = _edge_batch(rng, d, [(s, t) for s in edges for t in edges], 200000, lo=5, hi=40)
    empties = _edge_batch(rng, d, [(40, 45), (3, 100), (100, 3), (7, 0), (0, 7)], 200000,
                          empty_frac=0.3)
    longs = _edge_batch(rng, d, [(20, 70), (70, 20), (33, 33)], 200000, lo=200, hi=1024)

    def rand_doc(n_sent, lo, hi):
        lens = rng.integers(lo, hi + 1, n_sent)
        off = np.zeros(n_sent + 1, np.int32)
        np.cumsum(lens, out=off[1:])
        return off, rng.integers(0, 200000, int(off[-1])).astype(np.int32)
    wide = synth.pack_docs([rand_doc(120, 5, 40), rand_doc(700, 15, 25),     # ~14,000 distinct
                            rand_doc(60, 5, 40), rand_doc(1000, 25, 35),     # ~28,000: token-keyed
                            # at most 160 target sentences with 4,097-6,144 distinct
                            # tokens: the small-article preparation, the score launch
                            # of larger articles (from k_order's list)
                            rand_doc(40, 5, 40), rand_doc(100, 50, 60)])     # ~5,400
    dh = ctx.dict_create(d)
    od = O.OracleDict(d)
    for name, b in (("lognormal", w.batch), ("edges", edge), ("empties", empties), ("long", longs),
                    ("wide", wide)):
        got = ctx.score_q16(dh, b)
        assert len(got) == b.n_pairs
        for p in range(b.n_pairs):
            want = O.score_matrix(od, *b.pair(p))
            assert got[p].shape == want.shape, (name, p)
            if want.size:
                bad = np.argwhere(got[p] != want)
                assert bad.size == 0, f"{name} pair {p}: {len(bad)} cells differ, first {bad[:4].tolist()}"


def test_pinned_host_inputs(ctx):
    """The host-buffer call with pinned inputs and outputs (as the benchmark
    makes it), twice in a row: results as the oracle's, on lognormal pairs, on
    a pair whose target article has between 8,192 and 16,384 distinct tokens
    (the extra-wide launches) and on one with more (the token-keyed path)."""
    torch = pytest.importorskip("torch")
    w = synth.workload(2, n_pairs=200)
    rng = np.random.default_rng(83)
    docs = [w.batch.doc(d) for d in range(2 * w.batch.n_pairs)]
    def rand_doc(n_sent, lo, hi):
        lens = rng.integers(lo, hi + 1, n_sent)
        off = np.zeros(n_sent + 1, np.int32)
        np.cumsum(lens, out=off[1:])
        return off, rng.integers(0, 200000, int(off[-1])).astype(np.int32)
    docs += [rand_doc(120, 5, 40), rand_doc(700, 15, 25)]     # about 14,000 distinct target tokens
    docs += [rand_doc(60, 5, 40), rand_doc(1000, 25, 35)]     # about 28,000: the token-keyed path
    b = synth.pack_docs(docs)
    wb = synth.Workload("pinned", b, w.dictionary, [], [], w.settings + [(-16384, 16384)])
    want = oracle_results(wb)
    dh = ctx.dict_create(w.dictionary)
    P, n = b.n_pairs, len(wb.settings)
    pin_sent = torch.from_numpy(b.sent_off.copy()).pin_memory()
    pin_tok = torch.from_numpy(b.tokens.copy()).pin_memory()
    do = np.ascontiguousarray(b.doc_off)
    g = np.asarray([s[0] for s in wb.settings], np.int32)
    th = np.asarray([s[1] for s in wb.settings], np.int32)
    bc = mine.BatchC(P, b.sent_off.shape[0] - 1, b.tokens.shape[0], mine._ptr(do), pin_sent.data_ptr(),
                     pin_tok.data_ptr())
    sc = mine.SettingsC(n, mine._ptr(g), mine._ptr(th))
    S, T = b.sizes()
    cap = int(n * np.minimum(S, T).sum())
    outs = (np.zeros(P * n, np.int32), np.zeros(P * n, np.int32), np.zeros(P * n + 1, np.int64),
            np.zeros((cap, 3), np.int32), cap)
    for _ in range(2):
        ctx.run_batch_raw(dh, bc, sc, outs)
        got = mine.unpack_results(P, n, *outs[:4])
        assert_same(got, want, "pinned inputs")


def test_device_batch_graph_replay(ctx):
    """Repeating a device-buffer batch replays its captured graph: every
    kernel runs again on the current contents of the input buffers, so new
    tokens in the same buffers give the new results; a host-buffer call in
    between, or per-kernel profiling, falls back to planning and launching."""
    torch = pytest.importorskip("torch")
    w = synth.workload(2, n_pairs=300)
    b = w.batch
    dh = ctx.dict_create(w.dictionary)
    dev = torch.device("cuda:0")
    sent = torch.from_numpy(b.sent_off).to(dev)
    tok = torch.from_numpy(b.tokens).to(dev)
    P, n = b.n_pairs, len(w.settings)
    S, T = b.sizes()
    cap = int(n * np.minimum(S, T).sum())
    nw = torch.zeros(P * n, dtype=torch.int32, device=dev)
    ns = torch.zeros(P * n, dtype=torch.int32, device=dev)
    sel = torch.zeros(cap * 3, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    base = np.zeros(P + 1, np.int64)
    np.cumsum(n * np.minimum(S, T), out=base[1:])

    def run_and_read():
        nw.zero_()
        ns.zero_()
        sel.zero_()
        c0 = ctx.launch_count()
        ctx.run_batch_device(dh, P, b.doc_off, sent, tok, int(b.sent_off.shape[0] - 1),
                             int(b.tokens.shape[0]), w.settings, nw, ns, sel, cap, stream)
        torch.cuda.synchronize()
        ctx.check()
        a, c, e = nw.cpu().numpy(), ns.cpu().numpy(), sel.cpu().numpy().reshape(-1, 3)
        got = [[(int(a[p]), [tuple(int(v) for v in t) for t in e[base[p]:base[p] + c[p]]])]
               for p in range(P)]
        return got, ctx.launch_count() - c0

    want = oracle_results(w)
    first, n0 = run_and_read()
    assert_same(first, want, "captured call")
    for k in range(2):
        again, n1 = run_and_read()
        assert_same(again, want, f"replay {k}")
        assert n1 == n0 > 0
    # new contents in the same buffers
    rng = np.random.default_rng(77)
    tok2 = b.tokens.copy()
    flip = rng.random(tok2.shape[0]) < 0.2
    tok2[flip] = rng.integers(0, 200000, int(flip.sum()), dtype=np.int32)
    b2 = synth.Batch(b.doc_off, b.sent_off, tok2)
    tok.copy_(torch.from_numpy(tok2))
    got2, _ = run_and_read()
    assert_same(got2, oracle_results(w, b2), "replay on new tokens")
    # a host-buffer call rewrites the context's scratch: the next call plans again
    assert_same(ctx.run_batch(dh, b2, w.settings), oracle_results(w, b2), "host call")
    got3, _ = run_and_read()
    assert_same(got3, oracle_results(w, b2), "after a host call")
    ctx.profile(True)
    got4, _ = run_and_read()
    ctx.profile(False)
    ctx.profile_read()
    assert_same(got4, oracle_results(w, b2), "profiled call")


def _edge_batch(rng, d, sizes, vocab, lo=5, hi=30, empty_frac=0.0):
    cdf = synth._zipf_cdf(vocab)
    S = np.array([s for s, _ in sizes])
    T = np.array([t for _, t in sizes])
    b = synth.make_pairs(rng, cdf, d, S, T, np.full(len(sizes), 0.6), lo, hi)
    if empty_frac:
        docs = []
        for dd in range(2 * b.n_pairs):
            so, tk = b.doc(dd)
            lens = np.diff(so)
            keep = rng.random(lens.shape[0]) >= empty_frac
            new_tok = np.concatenate([tk[so[k]:so[k + 1]] if keep[k] else tk[:0]
                                      for k in range(lens.shape[0])]) if lens.shape[0] else tk[:0]
            new_off = np.zeros(lens.shape[0] + 1, np.int64)
            np.cumsum(np.where(keep, lens, 0), out=new_off[1:])
            docs.append((new_off.astype(np.int32), new_tok))
        b = synth.pack_docs(docs)
    return b


def test_alignment_strategies_agree(ctx):
    """Every pair aligned one warp each where allowed, then by pipelines of
    2, 4 and 8 warps where the shape allows, then by the autotuned tables:
    the results never change."""
    w = synth.workload(2, n_pairs=300)
    dh = ctx.dict_create(w.dictionary)
    want = oracle_results(w)
    rng = np.random.default_rng(5)
    sizes = [(s, t) for s in (1, 7, 31, 32, 33, 64, 100) for t in (1, 5, 32, 33, 200, 511, 512, 700)]
    edge = _edge_batch(rng, w.dictionary, sizes, 200000, lo=5, hi=40)
    want_e = oracle_results(w, edge)
    old = ctx.align_strategy()
    try:
        for tab in ([0] * mine.ALIGN_BINS, [3] * mine.ALIGN_BINS, [4] * mine.ALIGN_BINS,
                    [1] * mine.ALIGN_BINS):
            ctx.align_strategy(tab)
            assert ctx.align_strategy() == tab
            assert_same(ctx.run_batch(dh, w.batch, w.settings), want, f"strategy {tab[0]}")
            assert_same(ctx.run_batch(dh, edge, w.settings), want_e, f"edge sizes, strategy {tab[0]}")
        ctx.align_strategy(old)
        tuned = ctx.autotune()
        assert all(v in (0, 1, 3, 4) for v in tuned[6:18])
        assert tuned[:6] == old[:6] and tuned[18:] == old[18:]
        assert_same(ctx.run_batch(dh, w.batch, w.settings), want, "tuned")
        ctx.align_strategy(old)
        tuned = ctx.autotune_batch(dh, w.batch)
        assert all(v in (-1, 0, 1, 3, 4) for v in tuned)
        assert_same(ctx.run_batch(dh, w.batch, w.settings), want, "tuned on the batch")
        # tuned with a sweep of settings (three distinct gaps per pair)
        sweep = w.settings + [(-16384, 16384), (0, 65536), (-16384, 40000)]
        tuned = ctx.autotune_batch(dh, w.batch, sweep)
        assert all(v in (-1, 0, 1, 2, 3, 4) for v in tuned)
        assert_same(ctx.run_batch(dh, w.batch, w.settings), want, "tuned on the batch and a sweep")
        with pytest.raises(mine.MineError):
            ctx.autotune_batch(dh, w.batch, [(1, 0)])            # gap > 0
    finally:
        ctx.align_strategy(old)


def test_strategy_table_file(ctx, tmp_path):
    """The tuned table kept across processes: saved to a JSON file and loaded
    back into a context; a malformed file is refused and changes nothing."""
    old = ctx.align_strategy()
    try:
        tab = [(-1, 0, 1, 2, 3, 4)[k % 6] for k in range(mine.ALIGN_BINS)]
        ctx.align_strategy(tab)
        path = tmp_path / "strategy.json"
        ctx.align_strategy_save(path)
        assert json.loads(path.read_text()) == {"format": "mine-align-strategy", "bins": tab}
        ctx.align_strategy(old)
        assert ctx.align_strategy_load(path) == tab
        path.write_text('{"format": "mine-align-strategy", "bins": [9]}')
        with pytest.raises(mine.MineError):
            ctx.align_strategy_load(path)
        assert ctx.align_strategy() == tab
    finally:
        ctx.align_strategy(old)


def test_single_precision_scores(ctx):
    """Float scores within 1e-5 of the exact-arithmetic oracle on both score
    paths (document ids, and the token-keyed path of a target article with
    more than 8192 distinct tokens), including empty sentences."""
    w = synth.workload(2, n_pairs=120)
    w1 = synth.workload(1)
    rng = np.random.default_rng(9)
    src = [[int(x) for x in rng.integers(0, 200000, 30)] for _ in range(40)]
    tgt = [[int(x) for x in rng.integers(0, 200000, 400)] for _ in range(30)]
    big = synth.docs_from_lists(src, tgt)
    edge = _edge_batch(rng, w.dictionary, [(1, 1), (33, 65), (64, 31), (5, 0), (0, 4)], 200000,
                       empty_frac=0.2)
    for dd, b in ((w.dictionary, w.batch), (w1.dictionary, w1.batch), (w.dictionary, big),
                  (w.dictionary, edge)):
        dh = ctx.dict_create(dd)
        got = ctx.score_f32(dh, b)
        od = O.OracleDict(dd)
        for p in range(b.n_pairs):
            want = O.score_matrix_f64(od, *b.pair(p))
            assert got[p].shape == want.shape
            if want.size:
                err = np.abs(got[p].astype(np.float64) - want).max()
                assert err <= 1e-5, (p, err)


def test_tile_boundaries_and_degenerate_shapes(ctx):
    rng = np.random.default_rng(77)
    d = synth.make_dictionary(rng, 5000, 3)
    edges = [0, 1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129]
    sizes = [(s, t) for s in edges for t in edges]
    w = synth.Workload("edges", _edge_batch(rng, d, sizes, 5000), d, [-65536], [32768],
                       [(-65536, 32768), (-20000, 0), (0, 65536), (-131072, 50000)])
    dh = ctx.dict_create(d)
    got = ctx.run_batch(dh, w.batch, w.settings)
    assert_same(got, oracle_results(w), "tile edges")


def test_empty_sentences_and_long_sentences(ctx):
    rng = np.random.default_rng(78)
    d = synth.make_dictionary(rng, 3000, 4)
    sizes = [(40, 45), (3, 100), (100, 3), (50, 50), (1, 1), (7, 0), (0, 7)]
    b = _edge_batch(rng, d, sizes, 3000, empty_frac=0.3)
    w = synth.Workload("empties", b, d, [], [], [(-65536, 32768), (-30000, 10000)])
    dh = ctx.dict_create(d)
    assert_same(ctx.run_batch(dh, b, w.settings), oracle_results(w), "empty sentences")
    # sentences up to the 1024-token limit (columns no longer fit 32 per block)
    b2 = _edge_batch(rng, d, [(20, 70), (70, 20), (33, 33)], 3000, lo=200, hi=1024)
    w2 = synth.Workload("long", b2, d, [], [], [(-65536, 32768)])
    assert_same(ctx.run_batch(dh, b2, w2.settings), oracle_results(w2), "long sentences")


def test_unusual_dictionaries(ctx):
    rng = np.random.default_rng(79)
    # up to 32 translations per key, many shared translations, unknown tokens
    V = 400
    m = {}
    for key in range(0, V, 2):          # odd IDs have no entry
        k = int(rng.integers(1, 33))
        m[key] = list(rng.choice(60, size=min(k, 60), replace=False))
    d = synth.dictionary_from_map(m)
    cdf = synth._zipf_cdf(V)
    b = synth.make_pairs(rng, cdf, synth.make_dictionary(rng, V, 2),
                         np.array([30, 64, 5]), np.array([41, 64, 90]), np.full(3, 0.5), 1, 60)
    w = synth.Workload("dict", b, d, [], [], [(-65536, 32768), (-8192, 40000)])
    dh = ctx.dict_create(d)
    assert_same(ctx.run_batch(dh, b, w.settings), oracle_results(w), "dense dictionary")
    # keys given in arbitrary order
    perm = rng.permutation(d.n_keys)
    cnt = np.diff(d.trans_off)
    off = np.zeros(d.n_keys + 1, np.int64)
    np.cumsum(cnt[perm], out=off[1:])
    tr = np.concatenate([d.trans[d.trans_off[k]:d.trans_off[k + 1]] for k in perm])
    d2 = synth.Dictionary(d.keys[perm].copy(), off.astype(np.int32), tr.astype(np.int32))
    dh2 = ctx.dict_create(d2)
    assert_same(ctx.run_batch(dh2, b, w.settings), oracle_results(w), "permuted keys")


def test_align_matrix_any_sign(ctx):
    rng = np.random.default_rng(80)
    for S, T in [(1, 1), (1, 57), (57, 1), (31, 33), (64, 65), (100, 37), (129, 128), (300, 310)]:
        for kind in range(3):
            if kind == 0:
                M = synth.random_matrix(rng, S, T, values=[0, 1, 2])      # many ties
                g, th = -1, 0
            elif kind == 1:
                M = synth.random_matrix(rng, S, T, lo=-65536, hi=65536)
                g, th = -int(rng.integers(0, 70000)), int(rng.integers(-65536, 65536))
            else:
                M = synth.random_matrix(rng, S, T, lo=0, hi=65536)
                g, th = -65536, 32768
            got = ctx.align_matrix(M, g, th)
            assert got == O.align(M, [(g, th)])[0], (S, T, kind)


def test_tiled_alignment_agrees(ctx):
    """Pairs cut into tiles of 256 x 512 cells over many CTAs (ragged last
    tiles, a tile row or column of one stripe or one score tile, ties, signed
    scores) give the oracle's results; so does a mined batch of large pairs."""
    rng = np.random.default_rng(21)
    old = ctx.align_strategy()
    try:
        ctx.align_strategy([2] * mine.ALIGN_BINS)
        sizes = [(257, 513), (300, 1000), (600, 600), (1000, 520), (513, 1025), (777, 1300),
                 (289, 545), (1024, 1024)]
        for S, T in sizes:
            for kind in range(3):
                if kind == 0:
                    M = synth.random_matrix(rng, S, T, values=[0, 1, 2])
                    g, th = -1, 0
                elif kind == 1:
                    M = synth.random_matrix(rng, S, T, lo=-65536, hi=65536)
                    g, th = -int(rng.integers(0, 70000)), int(rng.integers(-65536, 65536))
                else:
                    M = synth.random_matrix(rng, S, T, lo=0, hi=65536)
                    g, th = -65536, 32768
                got = ctx.align_matrix(M, g, th)
                assert got == O.align(M, [(g, th)])[0], (S, T, kind)
        w = synth.workload(2, n_pairs=4)
        sub = _edge_batch(rng, w.dictionary, [(300, 600), (520, 700), (257, 513), (40, 45)], 200000,
                          lo=5, hi=40)
        dh = ctx.dict_create(w.dictionary)
        assert_same(ctx.run_batch(dh, sub, w.settings), oracle_results(w, sub), "tiled batch")
    finally:
        ctx.align_strategy(old)


def test_align_matrix_textbook_cases(ctx):
    rng = np.random.default_rng(81)
    for _ in range(20):
        a = rng.integers(0, 4, rng.integers(1, 90))
        b = rng.integers(0, 4, rng.integers(1, 90))
        eq = a[:, None] == b[None, :]
        lcs = np.where(eq, 65536, 0).astype(np.int32)
        lev = np.where(eq, 0, -65536).astype(np.int32)
        assert ctx.align_matrix(lcs, 0, 0) == O.align(lcs, [(0, 0)])[0]
        assert ctx.align_matrix(lev, -65536, -1) == O.align(lev, [(-65536, -1)])[0]


def test_tuning_sweep_64_settings(ctx):
    w = synth.workload(4, n_pairs=400)
    dh = ctx.dict_create(w.dictionary)
    assert len(w.settings) == 64
    got = ctx.run_batch(dh, w.batch, w.settings)
    assert_same(got, oracle_results(w), w.name)
    # thresholds only filter one path per gap: selections nest
    for p in range(len(got)):
        for gi in range(8):
            sels = [set(got[p][gi * 8 + t][1]) for t in range(8)]
            assert all(sels[t + 1] <= sels[t] for t in range(7))


@pytest.mark.slow
def test_long_documents_4000x4000(ctx):
    w = synth.workload(3, n_pairs=2)
    dh = ctx.dict_create(w.dictionary)
    got = ctx.run_batch(dh, w.batch, w.settings)
    assert_same(got, oracle_results(w), w.name)


def test_serving_alone_and_in_the_mix():
    """Requests submitted in waves while earlier ones run: every result equals
    the oracle's and the same pair mined alone, and the served batches did
    overlap on the device (at least two on it at the same moment)."""
    import time
    ctx = mine.Context(device=0, max_batch_pairs=24, batch_window_us=100)
    w = synth.workload(5, n_pairs=300)
    b = w.batch
    S, T = b.sizes()
    dh = ctx.dict_create(w.dictionary)
    tickets = {}
    for p in range(b.n_pairs):
        src, tgt = b.pair(p)
        settings = w.settings if p % 7 else [(-65536, 32768), (-32768, 49152), (-65536, 0)]
        tickets[ctx.submit(dh, src, tgt, settings)] = (p, settings)
        if p % 25 == 24:
            time.sleep(0.0003)
    got = {}
    while len(got) < sum(len(s) for _, s in tickets.values()):
        for (t, k, status, nw, pairs, lat) in ctx.poll(256, 200000):
            assert status == 0
            assert lat > 0
            got[(t, k)] = (nw, pairs)
    od = O.OracleDict(w.dictionary)
    rng = np.random.default_rng(5)
    check = set(rng.choice(b.n_pairs, 40, replace=False).tolist()) | set(np.nonzero(S > 100)[0].tolist())
    for t, (p, settings) in tickets.items():
        if p not in check:
            continue
        sub = b.subset([p])
        want, _ = O.mine_batch(od, sub, settings, THREADS)
        alone = ctx.run_batch(dh, sub, settings)
        for k in range(len(settings)):
            assert got[(t, k)] == want[0][k] == alone[0][k], (p, k)
    batches, overlap = ctx.serving_stats()
    ctx.close()
    assert batches >= 2
    assert overlap >= 2, f"{batches} batches, never two on the device at once"


def test_bounded_wait_runs_out_and_the_context_recovers(ctx):
    """Failure detection without a fault: the first warp of every warp
    pipeline withholds its rows (mine_test_inject, short waits), so the next
    warp's bounded wait runs out; the kernels return on their own, the call
    reports MINE_ETIMEDOUT, and the next call on the context mines exactly as
    the oracle does."""
    rng = np.random.default_rng(12)
    d = synth.make_dictionary(rng, 5000, 3)
    b = _edge_batch(rng, d, [(400, 400), (40, 45), (300, 600), (70, 33)], 5000)
    w = synth.Workload("pipeline", b, d, [], [], [(-65536, 32768)])
    dh = ctx.dict_create(d)
    want = oracle_results(w)
    old = ctx.align_strategy()
    try:
        ctx.align_strategy([1] * mine.ALIGN_BINS)   # a warp pipeline wherever the shape allows
        assert_same(ctx.run_batch(dh, b, w.settings), want, "warp pipelines")
        ctx.test_inject(mine.INJECT_WITHHOLD_ROWS, 1)
        with pytest.raises(mine.MineError) as e:
            ctx.run_batch(dh, b, w.settings)
        assert e.value.code == -5                     # MINE_ETIMEDOUT
        assert_same(ctx.run_batch(dh, b, w.settings), want, "after the timeout")
        ctx.test_inject(mine.INJECT_WITHHOLD_ROWS, 1)
        with pytest.raises(mine.MineError) as e:
            ctx.batch_wait(ctx.run_batch_async(dh, b, w.settings))
        assert e.value.code == -5
        assert_same(ctx.batch_wait(ctx.run_batch_async(dh, b, w.settings)), want, "asynchronous, after")
    finally:
        ctx.test_inject(mine.INJECT_WITHHOLD_ROWS, 0)
        ctx.align_strategy(old)


def test_errors_are_reported(ctx):
    w = synth.workload(1)
    dh = ctx.dict_create(w.dictionary)
    with pytest.raises(mine.MineError) as e:
        ctx.run_batch(dh, w.batch, [(1, 0)])                 # gap > 0
    assert e.value.code == -1
    with pytest.raises(mine.MineError) as e:
        ctx.run_batch(dh, w.batch, [(-1, 70000)])           # threshold > 1.0
    assert e.value.code == -1
    with pytest.raises(mine.MineError) as e:
        ctx.align_matrix(np.full((4000, 4000), 65536, np.int32), -1 << 20, 0)
    assert e.value.code == -4                              # H leaves int32
    bad = synth.Batch(w.batch.doc_off, w.batch.sent_off.copy(), w.batch.tokens.copy())
    bad.tokens[5] = 1 << 30                                 # token out of range
    with pytest.raises(mine.MineError):
        ctx.run_batch(dh, bad, w.settings)
    bad2 = synth.Batch(w.batch.doc_off, w.batch.sent_off.copy(), w.batch.tokens)
    bad2.sent_off[3] = bad2.sent_off[2] - 1                 # decreasing offsets
    with pytest.raises(mine.MineError):
        ctx.run_batch(dh, bad2, w.settings)
    # the context still works after rejected input
    assert ctx.run_batch(dh, w.batch, w.settings) == oracle_results(w)
    # duplicate dictionary keys
    d = synth.dictionary_from_map({1: [2], 3: [4]})
    d.keys[1] = 1
    with pytest.raises(mine.MineError):
        ctx.dict_create(d)


def test_budget_admission():
    w = synth.workload(1)
    src, tgt = w.batch.pair(0)
    with mine.Context(budget_bytes=4096) as small:
        dh = small.dict_create(w.dictionary)
        with pytest.raises(mine.MineError) as e:
            small.submit(dh, src, tgt, w.settings)
        assert e.value.code == -2
    with mine.Context(budget_bytes=1 << 22, max_inflight=2, max_batch_pairs=3) as c:
        dh = c.dict_create(w.dictionary)
        ts = [c.submit(dh, src, tgt, w.settings) for _ in range(20)]
        destroyed = False
        try:                                                # EBUSY while requests run
            c.dict_destroy(dh)
            destroyed = True
        except mine.MineError as e:
            assert e.code == -6
        out = []
        while len(out) < len(ts):
            out += c.poll(64, 100000)
        want = oracle_results(w)[0][0]
        assert all(o[2] == 0 and (o[3], o[4]) == want for o in out)
        if not destroyed:
            c.dict_destroy(dh)
