"""Thin Python binding of the miner's C ABI (include/mine.h).

Argument marshalling only: every step of the mining path runs in the CUDA
library.  Loading fails loudly when the compiled library is missing; there is
no CPU fallback.  PyTorch is used only to hand device buffers and streams to
the ``*_device`` entry point.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

MINE_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "EAGAIN", -4: "EOVERFLOW", -5: "ETIMEDOUT",
          -6: "EBUSY", -7: "ECUDA"}


class MineError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"mine error {ERRORS.get(code, code)}: {what}")


class Doc(ctypes.Structure):
    _fields_ = [("sent_off", ctypes.c_void_p), ("tokens", ctypes.c_void_p),
                ("n_sent", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("device", ctypes.c_int32), ("max_batch_pairs", ctypes.c_int32),
                ("batch_window_us", ctypes.c_int32)]


class Pair(ctypes.Structure):
    _fields_ = [("src_sent", ctypes.c_int32), ("tgt_sent", ctypes.c_int32),
                ("score", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("setting", ctypes.c_int32), ("nw_score", ctypes.c_int32),
                ("n_pairs", ctypes.c_int32), ("pairs", ctypes.POINTER(Pair)),
                ("latency_ns", ctypes.c_int64)]


class BatchC(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int32), ("n_sent", ctypes.c_int64),
                ("n_tok", ctypes.c_int64), ("doc_off", ctypes.c_void_p),
                ("sent_off", ctypes.c_void_p), ("tokens", ctypes.c_void_p)]


class SettingsC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("gaps", ctypes.c_void_p),
                ("thresholds", ctypes.c_void_p)]


# every function of include/mine.h with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int32
_L = ctypes.c_int64
SIGNATURES = {
    "mine_last_error": (ctypes.c_char_p, []),
    "mine_open": (_I, [ctypes.POINTER(Config), ctypes.POINTER(_P)]),
    "mine_close": (_I, [_P]),
    "mine_dict_create": (_I, [_P, _P, _P, _P, _I, ctypes.POINTER(_P)]),
    "mine_dict_destroy": (_I, [_P, _P]),
    "mine_submit": (_I, [_P, ctypes.POINTER(Doc), ctypes.POINTER(Doc), _P, _I, _I,
                         ctypes.POINTER(ctypes.c_uint64)]),
    "mine_submit_sweep": (_I, [_P, ctypes.POINTER(Doc), ctypes.POINTER(Doc), _P, _I, _P, _P,
                               ctypes.POINTER(ctypes.c_uint64)]),
    "mine_poll": (_I, [_P, ctypes.POINTER(Result), _I, _I]),
    "mine_result_free": (None, [_P, ctypes.POINTER(Result)]),
    "mine_align_matrix": (_I, [_P, _P, _I, _I, _I, _I, _P, ctypes.POINTER(_I),
                               ctypes.POINTER(_I)]),
    "mine_batch_capacity": (_L, [_P, _I, _I]),
    "mine_run_batch": (_I, [_P, _P, ctypes.POINTER(BatchC), ctypes.POINTER(SettingsC), _P, _P,
                            _P, _P, _L]),
    "mine_run_batch_async": (_I, [_P, _P, ctypes.POINTER(BatchC), ctypes.POINTER(SettingsC), _P,
                                  _P, _P, _P, _L, ctypes.POINTER(ctypes.c_uint64)]),
    "mine_batch_wait": (_I, [_P, ctypes.c_uint64]),
    "mine_run_batch_device": (_I, [_P, _P, ctypes.POINTER(BatchC), _P,
                                   ctypes.POINTER(SettingsC), _P, _P, _P, _L, _P]),
    "mine_check": (_I, [_P]),
    "mine_align_matrix_noalloc": (_I, [_P, _I, _I, _I, _I, _P, ctypes.POINTER(_I),
                                       ctypes.POINTER(_I), _P]),
    "mine_launch_count": (_L, [_P]),
    "mine_io_bytes": (_I, [_P, ctypes.POINTER(_L), ctypes.POINTER(_L)]),
    "mine_profile": (_I, [_P, _I]),
    "mine_profile_read": (_I, [_P, _P, _P, _I]),
    "mine_kernel_name": (ctypes.c_char_p, [_I]),
    "mine_autotune": (_I, [_P]),
    "mine_autotune_batch": (_I, [_P, _P, ctypes.POINTER(BatchC), ctypes.POINTER(SettingsC)]),
    "mine_score_f32": (_I, [_P, _P, ctypes.POINTER(BatchC), _P, _L]),
    "mine_score_q16": (_I, [_P, _P, ctypes.POINTER(BatchC), _P, _L]),
    "mine_test_inject": (_I, [_P, _I, _I]),
    "mine_serving_stats": (_I, [_P, ctypes.POINTER(_L), ctypes.POINTER(_I)]),
    "mine_int_peak": (_I, [_I, ctypes.POINTER(ctypes.c_double), _P, _I]),
    "mine_align_strategy": (_I, [_P, _P, _I, _I]),
    "mine_align_strategy_save": (_I, [_P, ctypes.c_char_p]),
    "mine_align_strategy_load": (_I, [_P, ctypes.c_char_p]),
    "mine_run_batch_bidi": (_I, [_P, _P, _P, ctypes.POINTER(BatchC), ctypes.POINTER(SettingsC), _P,
                                 _P, _P, _P, _P, _L]),
    "mine_tune_f1": (_I, [_P, _P, ctypes.POINTER(BatchC), ctypes.POINTER(SettingsC), _P, _P, _P,
                          ctypes.POINTER(_L), ctypes.POINTER(_I)]),
    "mine_best_match": (_I, [_P, _P, ctypes.POINTER(BatchC), _I, _P, _P, _P, _P, _L]),
}

ALIGN_BINS = 40
INJECT_CUDA_CALL = 1   # mine_test_inject kinds (include/mine.h)
INJECT_WITHHOLD_ROWS = 2

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmine.so (building it first if allowed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"the miner's CUDA library is not built: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def _c32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _check(rc, L=None):
    if rc < 0:
        L = L or load()
        raise MineError(rc, L.mine_last_error().decode(errors="replace"))
    return rc


def make_doc(sent_off, tokens):
    so, tk = _c32(sent_off), _c32(tokens)
    return Doc(_ptr(so), _ptr(tk), so.shape[0] - 1), (so, tk)


class AsyncBatch:
    """A call of ``Context.run_batch_async`` in flight: its ticket, and every
    array the library reads or writes until ``Context.batch_wait``."""

    def __init__(self, ticket, P, n, inputs, outs):
        self.ticket, self.P, self.n, self.inputs, self.outs = ticket, P, n, inputs, outs


class Context:
    """One miner context on one CUDA device."""

    def __init__(self, budget_bytes: int = 0, max_inflight: int = 0, device: int = -1,
                 max_batch_pairs: int = 0, batch_window_us: int = 0):
        self.L = load()
        cfg = Config(budget_bytes, max_inflight, device, max_batch_pairs, batch_window_us)
        h = ctypes.c_void_p()
        _check(self.L.mine_open(ctypes.byref(cfg), ctypes.byref(h)), self.L)
        self.h = h
        self._dicts = []

    def close(self):
        if getattr(self, "h", None):
            self.L.mine_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --------------------------------------------------------------- dictionary
    def dict_create(self, d):
        keys, off, tr = _c32(d.keys), _c32(d.trans_off), _c32(d.trans)
        h = ctypes.c_void_p()
        _check(self.L.mine_dict_create(self.h, _ptr(keys), _ptr(off), _ptr(tr),
                                       int(keys.shape[0]), ctypes.byref(h)), self.L)
        self._dicts.append(h)
        return h

    def dict_destroy(self, h):
        _check(self.L.mine_dict_destroy(self.h, h), self.L)
        self._dicts.remove(h)

    # --------------------------------------------------------------- batches
    def run_batch(self, dict_h, batch, settings):
        """Host buffers in and out.  Returns results[p][k] = (nw_score, [(i, j, s)])."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        P = (do.shape[0] - 1) // 2
        n = len(settings)
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        bc = BatchC(P, so.shape[0] - 1, tk.shape[0], _ptr(do), _ptr(so), _ptr(tk))
        sc = SettingsC(n, _ptr(g), _ptr(th))
        cap = max(int(self.L.mine_batch_capacity(_ptr(do), P, n)), 1)
        nw = np.zeros(P * n, np.int32)
        ns = np.zeros(P * n, np.int32)
        off = np.zeros(P * n + 1, np.int64)
        sel = np.zeros((cap, 3), np.int32)
        _check(self.L.mine_run_batch(self.h, dict_h, ctypes.byref(bc), ctypes.byref(sc),
                                     _ptr(nw), _ptr(ns), _ptr(off), _ptr(sel), cap), self.L)
        return unpack_results(P, n, nw, ns, off, sel)

    def run_batch_async(self, dict_h, batch, settings):
        """Enqueue a host-buffer call and return at once; ``batch_wait`` on the
        returned handle gives what ``run_batch`` would have returned.  The
        handle keeps every array of the call alive until then."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        P = (do.shape[0] - 1) // 2
        n = len(settings)
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        bc = BatchC(P, so.shape[0] - 1, tk.shape[0], _ptr(do), _ptr(so), _ptr(tk))
        sc = SettingsC(n, _ptr(g), _ptr(th))
        cap = max(int(self.L.mine_batch_capacity(_ptr(do), P, n)), 1)
        outs = (np.zeros(P * n, np.int32), np.zeros(P * n, np.int32), np.zeros(P * n + 1, np.int64),
                np.zeros((cap, 3), np.int32), cap)
        t = self.run_batch_async_raw(dict_h, bc, sc, outs)
        return AsyncBatch(t, P, n, (do, so, tk, g, th, bc, sc), outs)

    def batch_wait(self, handle):
        """Wait for a call of ``run_batch_async``; results[p][k] = (nw_score, [(i, j, s)])."""
        self.batch_wait_raw(handle.ticket)
        nw, ns, off, sel, _ = handle.outs
        return unpack_results(handle.P, handle.n, nw, ns, off, sel)

    def run_batch_async_raw(self, dict_h, bc, sc, outs):
        """Asynchronous host-buffer call with pre-built ctypes structs; returns its ticket."""
        nw, ns, off, sel, cap = outs
        t = ctypes.c_uint64()
        _check(self.L.mine_run_batch_async(self.h, dict_h, ctypes.byref(bc), ctypes.byref(sc), _ptr(nw),
                                           _ptr(ns), _ptr(off), _ptr(sel), cap, ctypes.byref(t)), self.L)
        return int(t.value)

    def batch_wait_raw(self, ticket):
        return _check(self.L.mine_batch_wait(self.h, ctypes.c_uint64(ticket)), self.L)

    def run_batch_bidi(self, fwd_h, bwd_h, batch, settings):
        """Both directions; results[p][k] = (nw forward, nw backward, union [(i, j, s)])."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        P = (do.shape[0] - 1) // 2
        n = len(settings)
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        bc = BatchC(P, so.shape[0] - 1, tk.shape[0], _ptr(do), _ptr(so), _ptr(tk))
        sc = SettingsC(n, _ptr(g), _ptr(th))
        cap = max(2 * int(self.L.mine_batch_capacity(_ptr(do), P, n)), 1)
        nwf = np.zeros(P * n, np.int32)
        nwb = np.zeros(P * n, np.int32)
        ns = np.zeros(P * n, np.int32)
        off = np.zeros(P * n + 1, np.int64)
        sel = np.zeros((cap, 3), np.int32)
        _check(self.L.mine_run_batch_bidi(self.h, fwd_h, bwd_h, ctypes.byref(bc), ctypes.byref(sc),
                                          _ptr(nwf), _ptr(nwb), _ptr(ns), _ptr(off), _ptr(sel), cap),
               self.L)
        res = []
        for p in range(P):
            row = []
            for k in range(n):
                r = p * n + k
                trip = sel[off[r]:off[r] + ns[r]]
                row.append((int(nwf[r]), int(nwb[r]), [tuple(int(v) for v in t) for t in trip]))
            res.append(row)
        return res

    def run_batch_bidi_raw(self, fwd_h, bwd_h, bc, sc, outs):
        """Bidirectional host-buffer call with pre-built ctypes structs (benchmark path)."""
        nwf, nwb, ns, off, sel, cap = outs
        return _check(self.L.mine_run_batch_bidi(self.h, fwd_h, bwd_h, ctypes.byref(bc),
                                                 ctypes.byref(sc), _ptr(nwf), _ptr(nwb), _ptr(ns),
                                                 _ptr(off), _ptr(sel), cap), self.L)

    def tune_f1(self, dict_h, batch, settings, truth):
        """Tuning objective over the settings: (tp, n_selected, n_truth, best)."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        P = (do.shape[0] - 1) // 2
        n = len(settings)
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        tr = _c32(truth)
        bc = BatchC(P, so.shape[0] - 1, tk.shape[0], _ptr(do), _ptr(so), _ptr(tk))
        sc = SettingsC(n, _ptr(g), _ptr(th))
        tp = np.zeros(n, np.int64)
        nsel = np.zeros(n, np.int64)
        nt = ctypes.c_int64()
        best = ctypes.c_int32()
        _check(self.L.mine_tune_f1(self.h, dict_h, ctypes.byref(bc), ctypes.byref(sc), _ptr(tr),
                                   _ptr(tp), _ptr(nsel), ctypes.byref(nt), ctypes.byref(best)), self.L)
        return [int(v) for v in tp], [int(v) for v in nsel], int(nt.value), int(best.value)

    def best_match(self, dict_h, batch, threshold):
        """Contrast without the path constraint: [(selection [(i, j, s)], repeated)] per pair."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        P = (do.shape[0] - 1) // 2
        bc = BatchC(P, so.shape[0] - 1, tk.shape[0], _ptr(do), _ptr(so), _ptr(tk))
        cap = max(int(so.shape[0] - 1), 1)
        ns = np.zeros(P, np.int32)
        rep = np.zeros(P, np.int32)
        off = np.zeros(P + 1, np.int64)
        sel = np.zeros((cap, 3), np.int32)
        _check(self.L.mine_best_match(self.h, dict_h, ctypes.byref(bc), int(threshold), _ptr(ns), _ptr(rep),
                                      _ptr(off), _ptr(sel), cap), self.L)
        return [([tuple(int(v) for v in t) for t in sel[off[p]:off[p] + ns[p]]], int(rep[p]))
                for p in range(P)]

    def run_batch_raw(self, dict_h, bc, sc, outs):
        """Host-buffer call with pre-built ctypes structs (benchmark path)."""
        nw, ns, off, sel, cap = outs
        return _check(self.L.mine_run_batch(self.h, dict_h, ctypes.byref(bc), ctypes.byref(sc),
                                            _ptr(nw), _ptr(ns), _ptr(off), _ptr(sel), cap),
                      self.L)

    def run_batch_device(self, dict_h, n_pairs, doc_off_host, sent_off_dev, tokens_dev,
                         n_sent, n_tok, settings, nw_dev, nsel_dev, sel_dev, sel_cap,
                         stream=None):
        """Device buffers (torch tensors or raw pointers) in and out, enqueued on stream."""
        def dp(x):
            return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
        do = _c32(doc_off_host)
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        bc = BatchC(n_pairs, n_sent, n_tok, ctypes.c_void_p(0), dp(sent_off_dev), dp(tokens_dev))
        sc = SettingsC(len(settings), _ptr(g), _ptr(th))
        st = ctypes.c_void_p(stream if isinstance(stream, int) else
                             (stream.cuda_stream if stream is not None else 0))
        return _check(self.L.mine_run_batch_device(self.h, dict_h, ctypes.byref(bc), _ptr(do),
                                                   ctypes.byref(sc), dp(nw_dev), dp(nsel_dev),
                                                   dp(sel_dev), int(sel_cap), st), self.L)

    def check(self):
        return _check(self.L.mine_check(self.h), self.L)

    def launch_count(self) -> int:
        return int(self.L.mine_launch_count(self.h))

    def io_bytes(self):
        """(host->device, device->host) bytes moved by run_batch calls so far."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self.L.mine_io_bytes(self.h, ctypes.byref(a), ctypes.byref(b)), self.L)
        return a.value, b.value

    def test_inject(self, kind: int, count: int):
        """Fault injection for tests (mine_test_inject)."""
        _check(self.L.mine_test_inject(self.h, int(kind), int(count)), self.L)

    def profile(self, enable: bool = True):
        _check(self.L.mine_profile(self.h, 1 if enable else 0), self.L)

    def score_f32(self, dict_h, batch):
        """Single-precision score matrices of every pair (list of S x T float32 arrays)."""
        return self._scores(dict_h, batch, np.float32, self.L.mine_score_f32)

    def score_q16(self, dict_h, batch):
        """Fixed-point (Q16) score matrices of every pair (list of S x T int32 arrays)."""
        return self._scores(dict_h, batch, np.int32, self.L.mine_score_q16)

    def _scores(self, dict_h, batch, dtype, fn):
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        S, T = batch.sizes()
        cells = int((S * T).sum())
        out = np.zeros(max(cells, 1), dtype)
        bc = BatchC(batch.n_pairs, int(so.shape[0] - 1), int(tk.shape[0]), _ptr(do), _ptr(so), _ptr(tk))
        _check(fn(self.h, dict_h, ctypes.byref(bc), _ptr(out), cells), self.L)
        res, o = [], 0
        for p in range(batch.n_pairs):
            n = int(S[p] * T[p])
            res.append(out[o:o + n].reshape(int(S[p]), int(T[p])))
            o += n
        return res

    def autotune(self):
        """Time the pipeline widths per size bin on this GPU and keep the
        fastest; returns the strategy table."""
        _check(self.L.mine_autotune(self.h), self.L)
        return self.align_strategy()

    def autotune_batch(self, dict_h, batch, settings=None):
        """Tune the per-bin alignment strategy on a batch of the workload and
        the settings it will be mined with (None: one default setting);
        returns the strategy table."""
        do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
        bc = BatchC(batch.n_pairs, int(so.shape[0] - 1), int(tk.shape[0]), _ptr(do), _ptr(so), _ptr(tk))
        sc = None
        if settings is not None:
            g = _c32([s[0] for s in settings])
            th = _c32([s[1] for s in settings])
            sc = SettingsC(len(settings), _ptr(g), _ptr(th))
        _check(self.L.mine_autotune_batch(self.h, dict_h, ctypes.byref(bc),
                                          ctypes.byref(sc) if sc is not None else None), self.L)
        return self.align_strategy()

    def align_strategy(self, table=None):
        """Get (table None) or set the per-bin strategy table: 0 one warp, 3 / 4 / 1
        pipelines of 2 / 4 / 8 warps, 2 tiles over many CTAs, -1 built-in rule
        (each where the pair's shape allows, else the nearest form)."""
        t = np.full(ALIGN_BINS, -1, np.int8) if table is None else np.ascontiguousarray(table, np.int8)
        _check(self.L.mine_align_strategy(self.h, _ptr(t), int(t.shape[0]), 1 if table is None else 0),
               self.L)
        return [int(v) for v in t]

    def align_strategy_save(self, path):
        """Write the strategy table to a JSON file (mine_align_strategy_save)."""
        _check(self.L.mine_align_strategy_save(self.h, os.fsencode(path)), self.L)

    def align_strategy_load(self, path):
        """Read a table written by align_strategy_save into this context; returns it."""
        _check(self.L.mine_align_strategy_load(self.h, os.fsencode(path)), self.L)
        return self.align_strategy()

    def profile_read(self):
        """{kernel name: (total device ms, timed launches)} since the last read."""
        ms = np.zeros(32, np.float64)
        n = np.zeros(32, np.int64)
        k = _check(self.L.mine_profile_read(self.h, _ptr(ms), _ptr(n), 32), self.L)
        return {self.L.mine_kernel_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(k)}

    # --------------------------------------------------------------- alignment only
    def align_matrix(self, M, gap, threshold):
        M = _c32(M)
        S, T = M.shape
        out = (Pair * max(min(S, T), 1))()
        n = ctypes.c_int32()
        nw = ctypes.c_int32()
        _check(self.L.mine_align_matrix(self.h, _ptr(M), S, T, int(gap), int(threshold),
                                        ctypes.cast(out, ctypes.c_void_p), ctypes.byref(n),
                                        ctypes.byref(nw)), self.L)
        return nw.value, [(out[k].src_sent, out[k].tgt_sent, out[k].score) for k in range(n.value)]

    # --------------------------------------------------------------- serving
    def submit(self, dict_h, src, tgt, settings):
        (ds, ks), (dt, kt) = make_doc(*src), make_doc(*tgt)
        t = ctypes.c_uint64()
        g = _c32([s[0] for s in settings])
        th = _c32([s[1] for s in settings])
        _check(self.L.mine_submit_sweep(self.h, ctypes.byref(ds), ctypes.byref(dt), dict_h,
                                        len(settings), _ptr(g), _ptr(th), ctypes.byref(t)),
               self.L)
        return t.value

    def serving_stats(self):
        """(batches served, largest number of them on the device at once)."""
        nb, mo = ctypes.c_int64(), ctypes.c_int32()
        _check(self.L.mine_serving_stats(self.h, ctypes.byref(nb), ctypes.byref(mo)), self.L)
        return int(nb.value), int(mo.value)

    def poll(self, max_out=1024, timeout_us=0):
        """[(ticket, setting, status, nw_score, [(i, j, s)], latency_ns)]"""
        buf = (Result * max_out)()
        n = _check(self.L.mine_poll(self.h, buf, max_out, int(timeout_us)), self.L)
        out = []
        for k in range(n):
            r = buf[k]
            pairs = [(r.pairs[q].src_sent, r.pairs[q].tgt_sent, r.pairs[q].score)
                     for q in range(r.n_pairs)]
            out.append((r.ticket, r.setting, r.status, r.nw_score, pairs, r.latency_ns))
            self.L.mine_result_free(self.h, ctypes.byref(buf[k]))
        return out


def align_matrix_noalloc(M, gap, threshold, stream=None):
    """Alignment of a host matrix without device allocation (current device).

    Returns (nw_score, [(i, j, s)]) like Context.align_matrix."""
    L = load()
    M = _c32(M)
    S, T = M.shape
    out = (Pair * max(min(S, T), 1))()
    n = ctypes.c_int32()
    nw = ctypes.c_int32()
    st = ctypes.c_void_p(stream if isinstance(stream, int) else
                         (stream.cuda_stream if stream is not None else 0))
    _check(L.mine_align_matrix_noalloc(_ptr(M), S, T, int(gap), int(threshold),
                                       ctypes.cast(out, ctypes.c_void_p), ctypes.byref(n),
                                       ctypes.byref(nw), st), L)
    return nw.value, [(out[k].src_sent, out[k].tgt_sent, out[k].score) for k in range(n.value)]


def int_peak(device: int = -1):
    """Measured int32 add/max rate of the device: (ops/s, [ops/s per form])."""
    L = load()
    best = ctypes.c_double()
    forms = np.zeros(3, np.float64)
    _check(L.mine_int_peak(int(device), ctypes.byref(best), _ptr(forms), 3), L)
    return float(best.value), [float(v) for v in forms]


def unpack_results(P, n, nw, ns, off, sel):
    res = []
    for p in range(P):
        row = []
        for k in range(n):
            r = p * n + k
            trip = sel[off[r]:off[r] + ns[r]]
            row.append((int(nw[r]), [tuple(int(v) for v in t) for t in trip]))
        res.append(row)
    return res
