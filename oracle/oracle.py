"""Python face of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this module.  It loads ``mine_oracle.c`` (compiled by
:func:`build`) through ctypes and adds two pure-Python pieces that are NOT the
recurrence: a brute-force enumerator of every monotone alignment (the paper's
"paths cannot go upward or leftward", Section 4) and the canonical-path rule,
used to pin the oracle's dynamic programme on tiny inputs.  Bidirectional
mining (the union of the two directions' selections), the tuning objective
(F1 against known translation pairs) and the contrast without the path
constraint (each source sentence's best target) are plain Python as well.

Parity pins for every function here live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

DIAG, UP, LEFT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "mine_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP when available) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path: str):
    """A ctypes handle on a compiled oracle library at ``path``."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32 = ctypes.c_int32
    L.oracle_dict_new.restype = P
    L.oracle_dict_new.argtypes = [P, P, P, i32]
    L.oracle_dict_free.argtypes = [P]
    L.oracle_score_matrix.argtypes = [P, P, P, i32, P, P, i32, P]
    L.oracle_score_matrix_f64.argtypes = [P, P, P, i32, P, P, i32, P]
    L.oracle_nw.restype = ctypes.c_int64
    L.oracle_nw.argtypes = [P, i32, i32, i32, P, P]
    L.oracle_traceback.restype = i32
    L.oracle_traceback.argtypes = [P, i32, i32, P]
    L.oracle_select.restype = i32
    L.oracle_select.argtypes = [P, i32, i32, P, i32, i32, P]
    L.oracle_align.argtypes = [P, i32, i32, i32, P, P, P, P, P]
    L.oracle_mine_batch.restype = i32
    L.oracle_mine_batch.argtypes = [P, i32, P, P, P, i32, P, P, P, P, P, P, i32]
    return L


def lib():
    """The oracle library (built on first use)."""
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class OracleDict:
    """The dictionary as the oracle holds it (sorted keys, bisection lookup)."""

    def __init__(self, d, L=None):
        self.L = L or lib()
        self._keep = (_c32(d.keys), _c32(d.trans_off), _c32(d.trans))
        k, o, t = self._keep
        self.h = self.L.oracle_dict_new(_p(k), _p(o), _p(t), int(k.shape[0]))

    def __del__(self):
        if getattr(self, "h", None):
            self.L.oracle_dict_free(self.h)
            self.h = None


def score_matrix(od: OracleDict, src, tgt) -> np.ndarray:
    """M[i, j] = fixed-point pair score of source sentence i, target j."""
    so, st = _c32(src[0]), _c32(src[1])
    to, tt = _c32(tgt[0]), _c32(tgt[1])
    S, T = so.shape[0] - 1, to.shape[0] - 1
    M = np.zeros((S, T), np.int32)
    od.L.oracle_score_matrix(od.h, _p(so), _p(st), S, _p(to), _p(tt), T, _p(M))
    return M


def score_matrix_f64(od: OracleDict, src, tgt) -> np.ndarray:
    """Real-valued pair score (exact division, double) of source sentence i,
    target j: the reference of the single-precision score."""
    so, st = _c32(src[0]), _c32(src[1])
    to, tt = _c32(tgt[0]), _c32(tgt[1])
    S, T = so.shape[0] - 1, to.shape[0] - 1
    M = np.zeros((S, T), np.float64)
    od.L.oracle_score_matrix_f64(od.h, _p(so), _p(st), S, _p(to), _p(tt), T, _p(M))
    return M


def nw(M, g: int, L=None):
    """(H[S][T], H, D) of the global alignment of M with gap g."""
    M = _c32(M)
    S, T = M.shape
    H = np.zeros((S + 1, T + 1), np.int64)
    D = np.zeros((S + 1, T + 1), np.uint8)
    r = (L or lib()).oracle_nw(_p(M), S, T, int(g), _p(H), _p(D))
    return int(r), H, D


def traceback(D, L=None) -> list:
    """Moves of the path from (S,T) back to (0,0) (first entry = last move)."""
    D = np.ascontiguousarray(D, np.uint8)
    S, T = D.shape[0] - 1, D.shape[1] - 1
    mv = np.zeros(S + T + 1, np.uint8)
    n = (L or lib()).oracle_traceback(_p(D), S, T, _p(mv))
    return [int(x) for x in mv[:n]]


def select(M, moves, theta: int, L=None) -> list:
    """[(i, j, s)] 0-based, DIAG steps with s > theta, increasing i."""
    M = _c32(M)
    S, T = M.shape
    mv = np.ascontiguousarray(np.asarray(moves, np.uint8))
    out = np.zeros((max(min(S, T), 1), 3), np.int32)
    n = (L or lib()).oracle_select(_p(M), S, T, _p(mv), int(mv.shape[0]), int(theta), _p(out))
    return [tuple(int(v) for v in row) for row in out[:n]]


def align(M, settings, L=None):
    """For each (gap, theta): (nw_score, [(i, j, s)])."""
    M = _c32(M)
    S, T = M.shape
    n = len(settings)
    g = _c32([s[0] for s in settings])
    th = _c32([s[1] for s in settings])
    cap = min(S, T)
    nws = np.zeros(n, np.int64)
    cnt = np.zeros(n, np.int32)
    sel = np.zeros((n, max(cap, 1), 3), np.int32)
    (L or lib()).oracle_align(_p(M), S, T, n, _p(g), _p(th), _p(nws), _p(cnt), _p(sel))
    return [(int(nws[k]), [tuple(int(v) for v in r) for r in sel[k, :cnt[k]]])
            for k in range(n)]


def mine_batch(od: OracleDict, batch, settings, threads: int = 1):
    """Whole path for every pair of a packed batch.

    Returns (results, threads_used); results[p][k] = (nw_score, [(i, j, s)])."""
    S, T = batch.sizes()
    P = batch.n_pairs
    n = len(settings)
    cap = np.minimum(S, T)
    base = np.zeros(P + 1, np.int64)
    np.cumsum(cap, out=base[1:])
    g = _c32([s[0] for s in settings])
    th = _c32([s[1] for s in settings])
    nws = np.zeros(P * n, np.int64)
    cnt = np.zeros(P * n, np.int32)
    sel = np.zeros(max(int(base[-1]) * n, 1) * 3, np.int32)
    do, so, tk = _c32(batch.doc_off), _c32(batch.sent_off), _c32(batch.tokens)
    used = od.L.oracle_mine_batch(od.h, P, _p(do), _p(so), _p(tk), n, _p(g), _p(th),
                                   _p(base), _p(nws), _p(cnt), _p(sel), int(threads))
    res = []
    for p in range(P):
        row = []
        for k in range(n):
            o = 3 * (int(base[p]) * n + k * int(cap[p]))
            c = int(cnt[p * n + k])
            trip = sel[o:o + 3 * c].reshape(-1, 3)
            row.append((int(nws[p * n + k]), [tuple(int(v) for v in r) for r in trip]))
        res.append(row)
    return res, int(used)


# ---------------------------------------------------------------------------
# bidirectional mining (Section 6, Table 2 "BI"; Section 7)
# ---------------------------------------------------------------------------

class _Packed:
    """A packed batch (doc_off, sent_off, tokens) built by the oracle itself."""

    def __init__(self, doc_off, sent_off, tokens):
        self.doc_off, self.sent_off, self.tokens = doc_off, sent_off, tokens

    @property
    def n_pairs(self) -> int:
        return (int(self.doc_off.shape[0]) - 1) // 2

    def sizes(self):
        d = self.doc_off.astype(np.int64)
        return d[1::2] - d[0:-1:2], d[2::2] - d[1::2]


def swap_roles(batch):
    """The same pairs with the two articles of every pair exchanged: the
    target article becomes the source (mining in the other direction)."""
    do = np.asarray(batch.doc_off, np.int64)
    so = np.asarray(batch.sent_off, np.int64)
    tk = np.asarray(batch.tokens, np.int32)
    doc_off, sent_off, toks = [0], [0], []
    for p in range(batch.n_pairs):
        for d in (2 * p + 1, 2 * p):
            for k in range(int(do[d]), int(do[d + 1])):
                toks.append(tk[int(so[k]):int(so[k + 1])])
                sent_off.append(sent_off[-1] + int(so[k + 1] - so[k]))
            doc_off.append(len(sent_off) - 1)
    tokens = np.concatenate(toks).astype(np.int32) if toks else np.zeros(0, np.int32)
    return _Packed(np.asarray(doc_off, np.int32), np.asarray(sent_off, np.int32), tokens)


def union_selection(fwd, bwd) -> list:
    """Union of the pairs one setting selects in the two directions.

    fwd holds (i, j, s) with i a source and j a target sentence; bwd holds
    (j, i, s') from mining with the roles exchanged (its first index is the
    target sentence).  A pair found in both directions appears once with the
    larger of its two scores; the result is ordered by (i, j)."""
    best = {}
    for i, j, s in fwd:
        best[(i, j)] = s
    for j, i, s in bwd:
        best[(i, j)] = max(best[(i, j)], s) if (i, j) in best else s
    return [(i, j, best[(i, j)]) for (i, j) in sorted(best)]


def mine_batch_bidi(od_fwd: OracleDict, od_bwd: OracleDict, batch, settings, threads: int = 1):
    """Mining with both dictionaries (source->target and target->source).

    Returns results[p][k] = (nw_score forward, nw_score backward,
    union of the two selections)."""
    fwd, _ = mine_batch(od_fwd, batch, settings, threads)
    bwd, _ = mine_batch(od_bwd, swap_roles(batch), settings, threads)
    return [[(fwd[p][k][0], bwd[p][k][0], union_selection(fwd[p][k][1], bwd[p][k][1]))
             for k in range(len(settings))] for p in range(batch.n_pairs)]


# ---------------------------------------------------------------------------
# tuning objective for Threshold and Penalty (Section 4; Section 6, Table 2
# "NWT"): F1 of the selected pairs against known translation pairs
# ---------------------------------------------------------------------------

def f1_counts(results, batch, truth):
    """Per setting k: (true positives, selected pairs) summed over the batch,
    and the number of known pairs.

    results[p][k] = (..., selection) with selection = [(i, j, s)] (the last
    entry of the tuple); truth[doc_off[2p] + i] = the target sentence that
    source sentence i of pair p translates, or -1.  A selected (i, j) is a
    true positive when truth says j for i."""
    do = np.asarray(batch.doc_off, np.int64)
    n = len(results[0]) if results else 0
    tp = [0] * n
    nsel = [0] * n
    for p, row in enumerate(results):
        s0 = int(do[2 * p])
        for k in range(n):
            sel = row[k][-1]
            nsel[k] += len(sel)
            tp[k] += sum(1 for (i, j, _) in sel if int(truth[s0 + i]) == j)
    n_truth = 0
    for p in range(len(results)):
        n_truth += sum(1 for i in range(int(do[2 * p]), int(do[2 * p + 1])) if int(truth[i]) >= 0)
    return tp, nsel, n_truth


def best_setting(tp, nsel, n_truth) -> int:
    """Index of the setting of highest F1 = 2 tp / (selected + known), exact
    rational comparison, the lowest index among equals; F1 = 0 when both
    counts are 0."""
    from fractions import Fraction
    f1 = [Fraction(2 * t, s + n_truth) if s + n_truth > 0 else Fraction(0)
          for t, s in zip(tp, nsel)]
    best = 0
    for k in range(1, len(f1)):
        if f1[k] > f1[best]:
            best = k
    return best


# ---------------------------------------------------------------------------
# contrast without the path constraint (Section 4: Yalign's A* search is not
# kept from going upward or leftward, so sentences can be matched again)
# ---------------------------------------------------------------------------

def best_match(M, theta):
    """Alignment without the constraint that paths cannot go upward or
    leftward, in its limit: a path may come back to any target sentence, so
    every source sentence i takes its best-scoring target j (the lowest j
    among equal scores), kept when s(i, j) > theta.

    Returns ([(i, j, s)] by increasing i, the number of target sentences
    taken by more than one source sentence)."""
    M = np.asarray(M)
    S = M.shape[0]
    sel = []
    for i in range(S):
        if M.shape[1] == 0:
            break
        row = [int(v) for v in M[i]]
        j = 0
        for c in range(1, len(row)):
            if row[c] > row[j]:
                j = c
        if row[j] > theta:
            sel.append((i, j, row[j]))
    taken = {}
    for _, j, _ in sel:
        taken[j] = taken.get(j, 0) + 1
    return sel, sum(1 for c in taken.values() if c > 1)


def best_match_batch(od: OracleDict, batch, theta):
    """best_match of every pair's score matrix: [(selection, repeated)]."""
    out = []
    for p in range(batch.n_pairs):
        do = np.asarray(batch.doc_off, np.int64)
        so = np.asarray(batch.sent_off, np.int64)
        tk = np.asarray(batch.tokens, np.int32)
        docs = []
        for d in (2 * p, 2 * p + 1):
            o = so[do[d]:do[d + 1] + 1]
            docs.append(((o - o[0]).astype(np.int32), tk[int(o[0]):int(o[-1])]))
        out.append(best_match(score_matrix(od, docs[0], docs[1]), theta))
    return out


# ---------------------------------------------------------------------------
# brute force (pure Python, tiny inputs only): every monotone alignment
# ---------------------------------------------------------------------------

def brute_force(M, g: int):
    """Enumerate every monotone path (0,0)->(S,T) with steps DIAG (+1,+1),
    UP (+1,0), LEFT (0,+1).  Score = sum of M over DIAG targets + g per gap.

    Paths are visited backwards from (S,T) trying DIAG, then UP, then LEFT, so
    the first path reaching the best score is the one whose reversed move
    sequence is lexicographically smallest under DIAG < UP < LEFT.
    Returns (best_score, canonical reversed moves, number of paths)."""
    M = np.asarray(M, np.int64)
    S, T = M.shape
    best = [None, None]
    count = [0]
    moves = []

    def rec(i, j, acc):
        if i == 0 and j == 0:
            count[0] += 1
            if best[0] is None or acc > best[0]:
                best[0], best[1] = acc, list(moves)
            return
        if i > 0 and j > 0:
            moves.append(DIAG)
            rec(i - 1, j - 1, acc + int(M[i - 1, j - 1]))
            moves.pop()
        if i > 0:
            moves.append(UP)
            rec(i - 1, j, acc + g)
            moves.pop()
        if j > 0:
            moves.append(LEFT)
            rec(i, j - 1, acc + g)
            moves.pop()

    rec(S, T, 0)
    return best[0], best[1], count[0]


def delannoy(m: int, n: int) -> int:
    """Number of monotone lattice paths with steps (1,0), (0,1), (1,1)."""
    from math import comb
    return sum(comb(m, k) * comb(n, k) * 2 ** k for k in range(min(m, n) + 1))
