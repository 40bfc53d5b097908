"""Host-buffer batch calls in flight together (mine_run_batch_async and
mine_batch_wait): CUDA path vs CPU oracle, bit-exact.

Two calls at a time, each with its own buffers: results equal the oracle's
whatever the order of the waits, with pinned host arrays (the input copies
of one call overlap the kernels of the other) and with pageable ones; device
errors come back from the wait; the dictionary stays alive while a call uses
it; closing the context waits for what is in flight.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import mine, synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
EINVAL, EAGAIN, EBUSY = -1, -3, -6


@pytest.fixture(scope="module")
def ctx():
    c = mine.Context(device=0)
    yield c
    c.close()


def oracle_results(d, batch, settings):
    res, _ = O.mine_batch(O.OracleDict(d), batch, settings, THREADS)
    return res


def assert_same(got, want, what):
    assert len(got) == len(want), what
    bad = [p for p in range(len(got)) if got[p] != want[p]]
    assert not bad, f"{what}: {len(bad)} pairs differ, first {bad[:8]}"


def _edge_batch(d, seed):
    rng = np.random.default_rng(seed)
    edges = [0, 1, 31, 32, 33, 64, 65]
    sizes = [(s, t) for s in edges for t in edges] + [(300, 600), (520, 40)]
    S = np.array([s for s, _ in sizes])
    T = np.array([t for _, t in sizes])
    return synth.make_pairs(rng, synth._zipf_cdf(200000), d, S, T, np.full(len(sizes), 0.6), 5, 40)


def test_two_calls_in_flight_any_wait_order(ctx):
    w = synth.workload(2, n_pairs=300)
    e = _edge_batch(w.dictionary, 91)
    sweep = w.settings + [(-16384, 16384), (0, 65536)]
    dh = ctx.dict_create(w.dictionary)
    a = ctx.run_batch_async(dh, w.batch, w.settings)
    b = ctx.run_batch_async(dh, e, sweep)
    assert b.ticket != a.ticket
    # a third call before a wait is refused, and nothing of it runs
    with pytest.raises(mine.MineError) as err:
        ctx.run_batch_async(dh, w.batch, w.settings)
    assert err.value.code == EAGAIN
    got_b = ctx.batch_wait(b)                     # the later call first
    c = ctx.run_batch_async(dh, e, w.settings)    # its slot is free again
    got_a = ctx.batch_wait(a)
    got_c = ctx.batch_wait(c)
    assert_same(got_a, oracle_results(w.dictionary, w.batch, w.settings), "first call")
    assert_same(got_b, oracle_results(w.dictionary, e, sweep), "second call, three settings")
    assert_same(got_c, oracle_results(w.dictionary, e, w.settings), "third call")
    # the synchronous call between them gives the same
    assert ctx.run_batch(dh, e, w.settings) == got_c
    # tickets are waited for once
    for t in (a.ticket, 0, 1 << 40):
        with pytest.raises(mine.MineError) as err:
            ctx.batch_wait_raw(t)
        assert err.value.code == EINVAL


def test_pinned_pipeline(ctx):
    """Calls of the benchmark's form (pinned inputs and outputs), two in
    flight all the time, on lognormal pairs and on pairs that take the
    extra-wide and the token-keyed paths: every call's results are the
    oracle's."""
    torch = pytest.importorskip("torch")
    w = synth.workload(2, n_pairs=200)
    rng = np.random.default_rng(92)
    docs = [w.batch.doc(d) for d in range(2 * w.batch.n_pairs)]

    def rand_doc(n_sent, lo, hi):
        lens = rng.integers(lo, hi + 1, n_sent)
        off = np.zeros(n_sent + 1, np.int32)
        np.cumsum(lens, out=off[1:])
        return off, rng.integers(0, 200000, int(off[-1])).astype(np.int32)

    docs += [rand_doc(120, 5, 40), rand_doc(700, 15, 25)]     # about 14,000 distinct target tokens
    docs += [rand_doc(60, 5, 40), rand_doc(1000, 25, 35)]     # about 28,000
    b = synth.pack_docs(docs)
    settings = w.settings + [(-16384, 16384)]
    want = oracle_results(w.dictionary, b, settings)
    dh = ctx.dict_create(w.dictionary)
    P, n = b.n_pairs, len(settings)
    pin_sent = torch.from_numpy(b.sent_off.copy()).pin_memory()
    pin_tok = torch.from_numpy(b.tokens.copy()).pin_memory()
    do = np.ascontiguousarray(b.doc_off)
    g = np.asarray([s[0] for s in settings], np.int32)
    th = np.asarray([s[1] for s in settings], np.int32)
    bc = mine.BatchC(P, b.sent_off.shape[0] - 1, b.tokens.shape[0], mine._ptr(do), pin_sent.data_ptr(),
                     pin_tok.data_ptr())
    sc = mine.SettingsC(n, mine._ptr(g), mine._ptr(th))
    S, T = b.sizes()
    cap = int(n * np.minimum(S, T).sum())

    def pinned_outs():
        z = lambda k, dt: torch.zeros(k, dtype=dt).pin_memory().numpy()
        return (z(P * n, torch.int32), z(P * n, torch.int32), z(P * n + 1, torch.int64),
                z(cap * 3, torch.int32).reshape(cap, 3), cap)

    outs = [pinned_outs(), pinned_outs()]
    pending = []
    for k in range(6):
        if len(pending) == 2:
            t, o = pending.pop(0)
            ctx.batch_wait_raw(t)
            assert_same(mine.unpack_results(P, n, *o[:4]), want, "pinned pipeline")
            for x in o[:4]:
                x.fill(-7)                          # the next call must write them again
        o = outs[k % 2]
        pending.append((ctx.run_batch_async_raw(dh, bc, sc, o), o))
    for t, o in pending:
        ctx.batch_wait_raw(t)
        assert_same(mine.unpack_results(P, n, *o[:4]), want, "pinned pipeline")


def test_errors_come_back_from_the_wait(ctx):
    w = synth.workload(1)
    dh = ctx.dict_create(w.dictionary)
    # argument errors are reported by the call itself
    with pytest.raises(mine.MineError) as err:
        ctx.run_batch_async(dh, w.batch, [(1, 0)])
    assert err.value.code == EINVAL
    # a token out of range is found on the device: the wait reports it
    bad = synth.Batch(w.batch.doc_off, w.batch.sent_off.copy(), w.batch.tokens.copy())
    bad.tokens[5] = 1 << 30
    h = ctx.run_batch_async(dh, bad, w.settings)
    ok = ctx.run_batch_async(dh, w.batch, w.settings)
    with pytest.raises(mine.MineError) as err:
        ctx.batch_wait(h)
    assert err.value.code == EINVAL
    # the other call in flight is unaffected
    want = oracle_results(w.dictionary, w.batch, w.settings)
    assert ctx.batch_wait(ok) == want
    # an empty batch
    empty = synth.Batch(np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert ctx.batch_wait(ctx.run_batch_async(dh, empty, w.settings)) == []
    # the dictionary of a call in flight cannot be destroyed
    h = ctx.run_batch_async(dh, w.batch, w.settings)
    with pytest.raises(mine.MineError) as err:
        ctx.dict_destroy(dh)
    assert err.value.code == EBUSY
    assert ctx.batch_wait(h) == want
    ctx.dict_destroy(dh)


def test_close_waits_for_calls_in_flight():
    w = synth.workload(2, n_pairs=100)
    c = mine.Context(device=0)
    dh = c.dict_create(w.dictionary)
    handles = [c.run_batch_async(dh, w.batch, w.settings) for _ in range(2)]
    c.close()
    want = oracle_results(w.dictionary, w.batch, w.settings)
    for h in handles:
        nw, ns, off, sel, _ = h.outs
        assert mine.unpack_results(h.P, h.n, nw, ns, off, sel) == want


def test_injected_cuda_failure_waits_and_the_context_recovers(ctx):
    """A CUDA call that fails after the first input copy (faked on the host
    by mine_test_inject, the call not made) returns MINE_ECUDA from the
    synchronous and the asynchronous call, with nothing of the call left in
    flight; the next call on the context mines as the oracle does."""
    torch = pytest.importorskip("torch")
    w = synth.workload(2, n_pairs=120)
    want = oracle_results(w.dictionary, w.batch, w.settings)
    dh = ctx.dict_create(w.dictionary)
    b = w.batch
    P, n = b.n_pairs, len(w.settings)
    S, T = b.sizes()
    cap = int(n * np.minimum(S, T).sum())
    for sync, positions in ((True, (1, 2, 3, 4, 5, 8, 9)), (False, (1, 3, 4, 5, 6, 8, 13))):
        for at in positions:
            # pinned inputs and outputs: the copies really are asynchronous
            sent = torch.from_numpy(b.sent_off.copy()).pin_memory()
            tok = torch.from_numpy(b.tokens.copy()).pin_memory()
            do = np.ascontiguousarray(b.doc_off)
            g = np.asarray([s[0] for s in w.settings], np.int32)
            th = np.asarray([s[1] for s in w.settings], np.int32)
            bc = mine.BatchC(P, b.sent_off.shape[0] - 1, b.tokens.shape[0], mine._ptr(do),
                             sent.data_ptr(), tok.data_ptr())
            sc = mine.SettingsC(n, mine._ptr(g), mine._ptr(th))
            pins = [torch.zeros(P * n, dtype=torch.int32).pin_memory(),
                    torch.zeros(P * n, dtype=torch.int32).pin_memory(),
                    torch.zeros(P * n + 1, dtype=torch.int64).pin_memory(),
                    torch.zeros(3 * cap, dtype=torch.int32).pin_memory()]
            outs = tuple(x.numpy() for x in pins) + (cap,)
            ctx.test_inject(mine.INJECT_CUDA_CALL, at)
            with pytest.raises(mine.MineError) as e:
                if sync:
                    ctx.run_batch_raw(dh, bc, sc, outs)
                else:
                    ctx.run_batch_async_raw(dh, bc, sc, outs)
            assert e.value.code == -7, (sync, at)
            ctx.test_inject(mine.INJECT_CUDA_CALL, 0)
            # the failed call's buffers may go at once
            del sent, tok, outs, pins
            assert_same(ctx.run_batch(dh, b, w.settings), want, f"after a failure at {at}")
    got = ctx.batch_wait(ctx.run_batch_async(dh, b, w.settings))
    assert_same(got, want, "asynchronous call after the failures")
