"""Pins of the CPU oracle against things other than itself.

The paper prints no worked example and no intermediate value, so the oracle is
pinned by: values worked out by hand from the definitions (tests/golden), brute
force over every monotone alignment (Section 4: paths cannot go upward or
leftward), textbook special cases (LCS, Levenshtein), closed forms and
invariants.  The last test plants plausible mistakes in a copy of the oracle
and checks that these pins catch every one of them.
"""
import itertools
import json
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DIAG, UP, LEFT = O.DIAG, O.UP, O.LEFT


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _dict_from_json(m):
    return synth.dictionary_from_map({int(k): v for k, v in m.items()})


# ---------------------------------------------------------------- scoring pins

def check_score_hand_examples(L=None):
    for name in ("score_hand_example.json", "score_hand_example_2.json",
                 "score_hand_example_3.json"):
        g = _gold(name)
        od = O.OracleDict(_dict_from_json(g["dictionary"]), L)
        b = synth.docs_from_lists(g["src"], g["tgt"])
        M = O.score_matrix(od, *b.pair(0))
        assert M.tolist() == g["M"], name


def test_score_hand_examples():
    check_score_hand_examples()


def test_score_hand_example_full_path():
    g = _gold("score_hand_example.json")
    M = np.asarray(g["M"], np.int32)
    r, H, D = O.nw(M, g["gap"])
    assert r == g["nw_score"]
    assert H.tolist() == g["nw_H"]
    mv = O.traceback(D)
    assert [list(t) for t in O.select(M, mv, 32768)] == g["selected_theta_32768"]
    assert [list(t) for t in O.select(M, mv, 50000)] == g["selected_theta_50000"]


def check_score_closed_forms(L=None):
    # identical sentence with an identity dictionary: every feature is 1.0
    ident = synth.dictionary_from_map({t: [t] for t in range(1, 20)})
    od = O.OracleDict(ident, L)
    sent = [3, 5, 5, 7, 11, 3, 2]
    M = O.score_matrix(od, *synth.docs_from_lists([sent], [list(sent)]).pair(0))
    assert M[0, 0] == 65536
    # disjoint vocabularies: only the length term survives, 0.25 * min/max
    for L1, L2 in [(3, 7), (7, 3), (5, 5), (1, 9), (13, 4)]:
        src = [1 + (k % 5) for k in range(L1)]
        tgt = [100 + k for k in range(L2)]
        M = O.score_matrix(od, *synth.docs_from_lists([src], [tgt]).pair(0))
        q_l = (min(L1, L2) * 65536) // max(L1, L2)
        assert M[0, 0] == (16384 * q_l) >> 16, (L1, L2)
    # empty target sentence: no overlap and no length agreement -> 0
    M = O.score_matrix(od, *synth.docs_from_lists([[1, 2]], [[]]).pair(0))
    assert M[0, 0] == 0
    # two empty sentences count as equal length: 0.25
    M = O.score_matrix(od, *synth.docs_from_lists([[]], [[]]).pair(0))
    assert M[0, 0] == 16384
    # source made only of unknown tokens: target coverage 0, source coverage 0
    M = O.score_matrix(od, *synth.docs_from_lists([[500, 501]], [[500, 501]]).pair(0))
    assert M[0, 0] == 16384


def test_score_closed_forms():
    check_score_closed_forms()


def test_score_real_hand_example():
    g = _gold("score_real_hand_example.json")
    base = _gold(g["same_inputs_as"])
    od = O.OracleDict(_dict_from_json(base["dictionary"]))
    b = synth.docs_from_lists(base["src"], base["tgt"])
    M = O.score_matrix_f64(od, *b.pair(0))
    want = np.array([[n / d for n, d in row] for row in g["M_num_den"]])
    assert np.abs(M - want).max() < 1e-15


def test_score_real_closed_forms():
    ident = synth.dictionary_from_map({t: [t] for t in range(1, 20)})
    od = O.OracleDict(ident)
    sent = [3, 5, 5, 7, 11, 3, 2]
    assert O.score_matrix_f64(od, *synth.docs_from_lists([sent], [list(sent)]).pair(0))[0, 0] == 1.0
    for L1, L2 in [(3, 7), (7, 3), (5, 5), (1, 9), (13, 4)]:
        src = [1 + (k % 5) for k in range(L1)]
        tgt = [100 + k for k in range(L2)]
        v = O.score_matrix_f64(od, *synth.docs_from_lists([src], [tgt]).pair(0))[0, 0]
        assert abs(v - 0.25 * min(L1, L2) / max(L1, L2)) < 1e-15
    assert O.score_matrix_f64(od, *synth.docs_from_lists([[1, 2]], [[]]).pair(0))[0, 0] == 0.0
    assert O.score_matrix_f64(od, *synth.docs_from_lists([[]], [[]]).pair(0))[0, 0] == 0.25
    assert O.score_matrix_f64(od, *synth.docs_from_lists([[500, 501]], [[500, 501]]).pair(0))[0, 0] == 0.25


def test_score_real_matches_fixed_point_within_its_rounding():
    """The fixed-point score floors three ratios and one weighted sum: 65536
    times the exact score exceeds it by at least 0 and less than 2.375."""
    w = synth.workload(2, n_pairs=40)
    od = O.OracleDict(w.dictionary)
    for p in range(w.batch.n_pairs):
        src, tgt = w.batch.pair(p)
        Mq = O.score_matrix(od, src, tgt).astype(np.float64)
        Mr = O.score_matrix_f64(od, src, tgt) * 65536.0
        assert (Mr - Mq >= -1e-9).all() and (Mr - Mq < 2.375).all(), p


def test_score_ignores_dictionary_key_order_and_token_order():
    rng = np.random.default_rng(7)
    w = synth.workload(1)
    d = w.dictionary
    perm = rng.permutation(d.n_keys)
    cnt = np.diff(d.trans_off)
    new_off = np.zeros(d.n_keys + 1, np.int64)
    np.cumsum(cnt[perm], out=new_off[1:])
    new_tr = np.concatenate([d.trans[d.trans_off[k]:d.trans_off[k + 1]] for k in perm])
    d2 = synth.Dictionary(d.keys[perm].copy(), new_off.astype(np.int32), new_tr.astype(np.int32))
    src, tgt = w.batch.pair(0)
    M1 = O.score_matrix(O.OracleDict(d), src, tgt)
    M2 = O.score_matrix(O.OracleDict(d2), src, tgt)
    assert np.array_equal(M1, M2)
    # shuffling the tokens inside every sentence changes no set and no length
    so, st = src
    st2 = st.copy()
    for i in range(len(so) - 1):
        seg = st2[so[i]:so[i + 1]]
        rng.shuffle(seg)
    M3 = O.score_matrix(O.OracleDict(d), (so, st2), tgt)
    assert np.array_equal(M1, M3)


# ---------------------------------------------------------------- NW pins

def check_nw_hand_examples(L=None):
    g = _gold("nw_hand_examples.json")
    for ex in g["examples"]:
        M = np.asarray(ex["M"], np.int32)
        r, H, D = O.nw(M, ex["gap"], L)
        assert r == ex["nw_score"], ex["name"]
        assert H.tolist() == ex["H"], ex["name"]
        assert D.tolist() == ex["D"], ex["name"]
        assert O.traceback(D, L) == ex["reversed_moves"], ex["name"]
        for key in ex:
            if key.startswith("selected_theta_"):
                th = key[len("selected_theta_"):]
                th = -1 if th == "minus1" else int(th)
                got = [list(t) for t in O.select(M, O.traceback(D, L), th, L)]
                assert got == ex[key], (ex["name"], key)


def test_nw_hand_examples():
    check_nw_hand_examples()


def test_brute_force_enumerates_delannoy_many_paths():
    # the enumerator itself: path counts are the Delannoy numbers
    for S, T in [(1, 1), (2, 3), (3, 3), (4, 2), (5, 5)]:
        assert O.brute_force(np.zeros((S, T), np.int32), -1)[2] == O.delannoy(S, T)
    assert O.delannoy(7, 7) == 48639


def check_brute_force(L=None, sizes=None, reps=3, seed=1509):
    rng = np.random.default_rng(seed)
    sizes = sizes or [(S, T) for S in range(1, 6) for T in range(1, 6)]
    for S, T in sizes:
        for rep in range(reps):
            if rep % 3 == 0:      # many ties
                M = synth.random_matrix(rng, S, T, values=[0, 16384, 32768])
                g = int(rng.choice([0, -16384, -32768]))
            elif rep % 3 == 1:    # signed, few ties
                M = synth.random_matrix(rng, S, T, lo=-65536, hi=65536)
                g = -int(rng.integers(0, 65537))
            else:                 # non-negative scores as produced by the scorer
                M = synth.random_matrix(rng, S, T, lo=0, hi=65536)
                g = -int(rng.integers(0, 131073))
            best, canon, _ = O.brute_force(M, g)
            r, H, D = O.nw(M, g, L)
            assert r == best, (S, T, rep)
            assert O.traceback(D, L) == canon, (S, T, rep)


def test_brute_force_small():
    check_brute_force()


def test_brute_force_up_to_7():
    check_brute_force(sizes=[(6, 6), (7, 5), (5, 7), (7, 7)], reps=2, seed=1510)


def _lcs_brute(a, b):
    # longest subsequence of a that is also a subsequence of b, by enumeration
    def is_sub(x, y):
        it = iter(y)
        return all(c in it for c in x)
    for k in range(min(len(a), len(b)), -1, -1):
        for idx in itertools.combinations(range(len(a)), k):
            if is_sub([a[i] for i in idx], b):
                return k
    return 0


def _edit_brute(a, b):
    # shortest edit script by breadth-first search over (prefix, prefix) states
    from collections import deque
    seen = {(0, 0): 0}
    q = deque([(0, 0)])
    while q:
        i, j = q.popleft()
        d = seen[(i, j)]
        if i == len(a) and j == len(b):
            return d
        nxt = []
        if i < len(a) and j < len(b):
            nxt.append(((i + 1, j + 1), 0 if a[i] == b[j] else 1))
        if i < len(a):
            nxt.append(((i + 1, j), 1))
        if j < len(b):
            nxt.append(((i, j + 1), 1))
        for st, c in nxt:
            if c == 0 and (st not in seen or seen[st] > d):
                seen[st] = d
                q.appendleft(st)
            elif c == 1 and st not in seen:
                seen[st] = d + 1
                q.append(st)
    raise AssertionError


def _eq_matrix(a, b, hit, miss):
    return np.asarray([[hit if x == y else miss for y in b] for x in a], np.int32)


def check_textbook_special_cases(L=None, n=40, seed=11):
    g = _gold("nw_hand_examples.json")
    e, l = g["edit_distance"], g["lcs"]
    r, _, _ = O.nw(_eq_matrix(e["a"], e["b"], 0, -65536), -65536, L)
    assert -r // 65536 == e["distance"]
    r, _, _ = O.nw(_eq_matrix(l["a"], l["b"], 65536, 0), 0, L)
    assert r // 65536 == l["length"]
    rng = np.random.default_rng(seed)
    for _ in range(n):
        a = list(rng.integers(0, 3, rng.integers(1, 8)))
        b = list(rng.integers(0, 3, rng.integers(1, 8)))
        r, _, _ = O.nw(_eq_matrix(a, b, 65536, 0), 0, L)
        assert r == 65536 * _lcs_brute(a, b)
        r, _, _ = O.nw(_eq_matrix(a, b, 0, -65536), -65536, L)
        assert r == -65536 * _edit_brute(a, b)


def test_textbook_special_cases():
    check_textbook_special_cases()


def check_closed_forms(L=None, seed=3):
    rng = np.random.default_rng(seed)
    # single source sentence: either match exactly one target (best one) and
    # skip the other T-1, or skip all T and the source sentence itself
    for T in [1, 2, 5, 33]:
        M = synth.random_matrix(rng, 1, T, lo=0, hi=65536)
        for g in [0, -1000, -65536, -200000]:
            r, _, _ = O.nw(M, g, L)
            assert r == max(int(M.max()) + g * (T - 1), g * (T + 1))
    # zero matrix: |S-T| gaps; the canonical path matches from the end and
    # leaves the surplus sentences unmatched at the start
    for S, T in [(1, 4), (4, 1), (3, 3), (2, 7), (9, 4)]:
        g = -65536
        r, _, D = O.nw(np.zeros((S, T), np.int32), g, L)
        assert r == g * abs(S - T)
        mv = O.traceback(D, L)
        gap_move = LEFT if T > S else UP
        assert mv == [DIAG] * min(S, T) + [gap_move] * abs(S - T)


def test_closed_forms():
    check_closed_forms()


def _walk(mv, S, T):
    i, j = S, T
    cells = []
    for m in mv:
        if m == DIAG:
            cells.append((i, j))
            i, j = i - 1, j - 1
        elif m == UP:
            i -= 1
        else:
            j -= 1
        assert i >= 0 and j >= 0
    assert (i, j) == (0, 0)
    return cells[::-1]


def check_invariants(L=None, seed=5):
    rng = np.random.default_rng(seed)
    for S, T in [(50, 70), (70, 50), (1, 90), (64, 64), (33, 31)]:
        M = synth.random_matrix(rng, S, T, lo=0, hi=65536)
        for g in [0, -16384, -65536, -131072]:
            r, H, D = O.nw(M, g, L)
            mv = O.traceback(D, L)
            cells = _walk(mv, S, T)
            # score along the path equals the optimum
            assert r == sum(int(M[i - 1, j - 1]) for i, j in cells) + g * (len(mv) - len(cells))
            assert len(mv) - len(cells) == S + T - 2 * len(cells)
            # strictly increasing in both coordinates (each sentence once)
            assert all(a[0] < b[0] and a[1] < b[1] for a, b in zip(cells, cells[1:]))
            # the optimum does not depend on which article is called the source
            rt, _, _ = O.nw(np.ascontiguousarray(M.T), g, L)
            assert rt == r
            # thresholds only filter: selections nest
            prev = None
            for th in [0, 16384, 32768, 49152, 65536]:
                sel = set(O.select(M, mv, th, L))
                assert all(s > th for _, _, s in sel)
                if prev is not None:
                    assert sel <= prev
                prev = sel


def test_invariants():
    check_invariants()


def test_overflow_bound_holds_for_accepted_inputs():
    # (S+T)|g| + min(S,T)*65536 < 2^31 keeps every H inside int32
    S = T = 4000
    g = -131072
    assert (S + T) * abs(g) + min(S, T) * 65536 < 2 ** 31


# ------------------------------------------------ planted mistakes are caught

_MUTANTS = {
    "diag tie loses to up": ("(diag == best) ? OR_DIAG : (up == best) ? OR_UP : OR_LEFT",
                             "(up == best) ? OR_UP : (diag == best) ? OR_DIAG : OR_LEFT"),
    "up/left tie swapped": ("(diag == best) ? OR_DIAG : (up == best) ? OR_UP : OR_LEFT",
                            "(diag == best) ? OR_DIAG : (left == best) ? OR_LEFT : OR_UP"),
    "gap dropped from up": ("int64_t up = h[(i - 1) * W + j] + g;",
                            "int64_t up = h[(i - 1) * W + j];"),
    "transposed score index": ("M[(int64_t)(i - 1) * T + (j - 1)];\n            int64_t up",
                               "M[(int64_t)(j - 1) * T + (i - 1) < (int64_t)S * T ? (int64_t)(j - 1) * T + (i - 1) : 0];\n            int64_t up"),
    "free end gaps on first row": ("h[j] = (int64_t)j * g;", "h[j] = 0;"),
    "source/target counts swapped": ("int64_t q_t = tgt[j].m > 0 ? (a * 65536) / tgt[j].m : 0;",
                                     "int64_t q_t = src[i].n > 0 ? (a * 65536) / src[i].n : 0;"),
    "coverage from multiset": [("src[i].nu = sort_unique(src[i].U, w);",
                                "src[i].nu = w; qsort(src[i].U, (size_t)w, sizeof(int32_t), cmp_i32);"),
                               ("{ ++a; ++x; ++y; }", "{ ++a; ++x; }")],
    "length term weight swapped": ("int64_t s = (49152 * ((q_t + q_s) / 2) + 16384 * q_l) / 65536;",
                                   "int64_t s = (16384 * ((q_t + q_s) / 2) + 49152 * q_l) / 65536;"),
    "threshold not strict": ("if (s > theta) {", "if (s >= theta) {"),
    "unknown tokens not counted": ("src[i].n = sort_unique(src[i].X, L);",
                                   "src[i].n = sort_unique(src[i].X, L); { int32_t w2 = 0; for (int32_t p = 0; p < src[i].n; ++p) { const int32_t *tr; if (dict_lookup(d, src[i].X[p], &tr)) src[i].X[w2++] = src[i].X[p]; } src[i].n = w2; }"),
    "b counts translations not tokens": ("for (int32_t k = 0; k < c && !hit; ++k) hit = contains",
                                         "for (int32_t k = 0; k < c; ++k) hit += contains"),
}


def _run_all_pins(L):
    checks = [check_score_hand_examples, check_score_closed_forms, check_nw_hand_examples,
              lambda L: check_brute_force(L, reps=3), check_textbook_special_cases,
              check_closed_forms, check_invariants]
    failed = []
    for c in checks:
        try:
            c(L)
        except AssertionError:
            failed.append(c)
    return failed


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    edits = _MUTANTS[name]
    edits = edits if isinstance(edits, list) else [edits]
    src = open(O._SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation anchor for {name!r} not unique in the oracle"
        src = src.replace(old, new)
    path = tmp_path / "mutant.c"
    path.write_text(src)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(path), "-o", str(so)],
                   check=True, capture_output=True)
    L = O.load(str(so))
    assert _run_all_pins(L), f"no pin caught the planted mistake {name!r}"


def test_unmutated_oracle_passes_all_pins():
    assert _run_all_pins(O.lib()) == []


# ------------------------------------------- bidirectional mining and tuning pins
#
# Section 6 (Table 2, "BI") mines with classifiers trained in both directions
# and keeps what either finds; Section 4 tunes Threshold and Penalty (Table 2,
# "NWT").  The oracle's union of the two directions and its F1 objective are
# pinned by hand-worked examples, special cases and set identities; planted
# mistakes in a copy of the Python oracle must be caught.

def _dicts(c):
    f = synth.dictionary_from_map({int(k): v for k, v in c["fwd_dictionary"].items()})
    b = synth.dictionary_from_map({int(k): v for k, v in c["bwd_dictionary"].items()})
    return f, b


def check_bidi_hand_examples(m=O):
    g = _gold("bidi_hand_examples.json")
    st = [(g["gap"], g["theta"])]
    for c in g["cases"]:
        df, db = _dicts(c)
        of, ob = m.OracleDict(df), m.OracleDict(db)
        b = synth.docs_from_lists(c["src"], c["tgt"])
        sb = m.swap_roles(b)
        assert m.score_matrix(of, *b.pair(0)).tolist() == c["M_fwd"], c["name"]
        so = np.asarray(sb.sent_off)
        do = np.asarray(sb.doc_off)
        src = (so[do[0]:do[1] + 1] - so[do[0]], sb.tokens[so[do[0]]:so[do[1]]])
        tgt = (so[do[1]:do[2] + 1] - so[do[1]], sb.tokens[so[do[1]]:so[do[2]]])
        assert m.score_matrix(ob, src, tgt).tolist() == c["M_bwd"], c["name"]
        fw, _ = m.mine_batch(of, b, st)
        bw, _ = m.mine_batch(ob, sb, st)
        assert fw[0][0] == (c["nw_fwd"], [tuple(t) for t in c["sel_fwd"]]), c["name"]
        assert bw[0][0] == (c["nw_bwd"], [tuple(t) for t in c["sel_bwd"]]), c["name"]
        r = m.mine_batch_bidi(of, ob, b, st)
        assert r[0][0] == (c["nw_fwd"], c["nw_bwd"], [tuple(t) for t in c["union"]]), c["name"]


def test_bidi_hand_examples():
    check_bidi_hand_examples()


def _small_bidi_workload(n_pairs=10):
    w = synth.workload(2, n_pairs=n_pairs)
    return w, synth.reverse_dictionary(w.dictionary)


def check_bidi_exact_inverse_transposes(m=O):
    # with the exact inverse dictionary, a' = |U'_j ∩ X_i| counts the source
    # tokens that hit V_j (= b) and b' counts the target tokens some source
    # token translates to (= a), while m' = n_i and n' = m_j: the two coverage
    # terms exchange roles and the backward matrix is the transpose
    w = synth.workload(2, n_pairs=6)
    inv = synth.invert_dictionary(w.dictionary)
    of, ob = m.OracleDict(w.dictionary), m.OracleDict(inv)
    sb = m.swap_roles(w.batch)
    so, do = np.asarray(sb.sent_off), np.asarray(sb.doc_off)
    for p in range(w.batch.n_pairs):
        Mf = m.score_matrix(of, *w.batch.pair(p))
        src = (so[do[2 * p]:do[2 * p + 1] + 1] - so[do[2 * p]], sb.tokens[so[do[2 * p]]:so[do[2 * p + 1]]])
        tgt = (so[do[2 * p + 1]:do[2 * p + 2] + 1] - so[do[2 * p + 1]],
               sb.tokens[so[do[2 * p + 1]]:so[do[2 * p + 2]]])
        Mb = m.score_matrix(ob, src, tgt)
        assert np.array_equal(Mb, Mf.T), p
    r = m.mine_batch_bidi(of, ob, w.batch, [(-65536, 32768)])
    assert all(row[0][0] == row[0][1] for row in r)


def test_bidi_exact_inverse_transposes():
    check_bidi_exact_inverse_transposes()


def check_bidi_identities(m=O):
    w, inv = _small_bidi_workload()
    st = [(-65536, 32768), (-16384, 16384), (-131072, 49152)]
    of, ob = m.OracleDict(w.dictionary), m.OracleDict(inv)
    b = w.batch
    sb = m.swap_roles(b)
    # exchanging the roles twice gives the batch back
    bb = m.swap_roles(sb)
    for f in ("doc_off", "sent_off", "tokens"):
        assert np.array_equal(np.asarray(getattr(bb, f)), np.asarray(getattr(b, f)))
    S, T = b.sizes()
    S2, T2 = sb.sizes()
    assert np.array_equal(S, T2) and np.array_equal(T, S2)
    fw, _ = m.mine_batch(of, b, st)
    bw, _ = m.mine_batch(ob, sb, st)
    un = m.mine_batch_bidi(of, ob, b, st)
    for p in range(b.n_pairs):
        for k in range(len(st)):
            F = {(i, j): s for i, j, s in fw[p][k][1]}
            B = {(i, j): s for j, i, s in bw[p][k][1]}
            nf, nb, U = un[p][k]
            assert (nf, nb) == (fw[p][k][0], bw[p][k][0])
            keys = [(i, j) for i, j, _ in U]
            assert keys == sorted(set(keys)) and len(keys) == len(set(F) | set(B))
            assert set(keys) == set(F) | set(B)
            for i, j, s in U:
                assert s == max(F.get((i, j), -1), B.get((i, j), -1))
                assert s > st[k][1]
            # each direction's selection is a monotone chain: i and j increase together
            for sel in (sorted(F), sorted(B)):
                assert all(a[1] < c[1] for a, c in zip(sel, sel[1:]))


def test_bidi_identities():
    check_bidi_identities()


def check_bidi_special_cases(m=O):
    w, _ = _small_bidi_workload(6)
    st = [(-65536, 32768), (-32768, 20000)]
    of = m.OracleDict(w.dictionary)
    fw, _ = m.mine_batch(of, w.batch, st)
    # a reverse dictionary that translates nothing scores every backward cell
    # 0.25 q_l <= 16384: nothing above these thresholds, so the union is the
    # forward selection
    empty = synth.dictionary_from_map({})
    un = m.mine_batch_bidi(of, m.OracleDict(empty), w.batch, st)
    for p in range(w.batch.n_pairs):
        for k in range(len(st)):
            assert un[p][k][2] == fw[p][k][1]
    # one-sentence articles in both roles: the union holds (0, 0) exactly
    # when one direction scores it above the threshold
    b = synth.docs_from_lists([[1, 2]], [[11]])
    d1 = synth.dictionary_from_map({1: [11]})
    d2 = synth.dictionary_from_map({11: [1]})
    r = m.mine_batch_bidi(m.OracleDict(d1), m.OracleDict(d2), b, [(-65536, 0), (-65536, 65536)])
    assert r[0][0][2] and r[0][0][2][0][:2] == (0, 0) and r[0][1][2] == []


def test_bidi_special_cases():
    check_bidi_special_cases()


def check_f1_hand_example(m=O):
    g = _gold("f1_hand_example.json")
    b = synth.Batch(np.asarray(g["doc_off"], np.int32), np.zeros(11, np.int32), np.zeros(0, np.int32))
    res = [[(0, [tuple(t) for t in sel]) for sel in row] for row in g["selections"]]
    tp, nsel, nt = m.f1_counts(res, b, np.asarray(g["truth"], np.int32))
    assert (tp, nsel, nt) == (g["tp"], g["selected"], g["n_truth"])
    assert [[2 * t, s + nt] for t, s in zip(tp, nsel)] == g["f1_num_den"]
    assert m.best_setting(tp, nsel, nt) == g["best"]


def test_f1_hand_example():
    check_f1_hand_example()


def check_f1_closed_forms(m=O):
    w = synth.workload(2, n_pairs=8)
    st = [(-65536, 32768), (-16384, 16384), (-131072, 49152)]
    res, _ = m.mine_batch(m.OracleDict(w.dictionary), w.batch, st)
    do = w.batch.doc_off
    for k in range(len(st)):
        # known pairs = exactly what setting k selects: F1 = 1 there
        truth = np.full(int(do[-1]), -1, np.int32)
        for p in range(w.batch.n_pairs):
            for i, j, _ in res[p][k][1]:
                truth[int(do[2 * p]) + i] = j
        tp, nsel, nt = m.f1_counts(res, w.batch, truth)
        assert tp[k] == nsel[k] == nt
        best = m.best_setting(tp, nsel, nt)
        assert 2 * tp[best] == nsel[best] + nt and best <= k
    # nothing known: every F1 is 0 and the first setting is best
    none = np.full(int(do[-1]), -1, np.int32)
    tp, nsel, nt = m.f1_counts(res, w.batch, none)
    assert tp == [0, 0, 0] and nt == 0 and m.best_setting(tp, nsel, nt) == 0
    # nothing selected and nothing known: F1 counts as 0
    assert m.best_setting([0, 0], [0, 0], 0) == 0
    # the generator's planted pairs: each known pair is one source sentence
    tr = synth.truth_of(w.batch, w.planted)
    _, _, nt = m.f1_counts(res, w.batch, tr)
    assert nt == w.planted.shape[0]


def test_f1_closed_forms():
    check_f1_closed_forms()


_PY_MUTANTS = {
    "union without the role exchange": ("    for j, i, s in bwd:\n", "    for i, j, s in bwd:\n"),
    "union keeps the forward score": ("best[(i, j)] = max(best[(i, j)], s) if (i, j) in best else s",
                                      "best[(i, j)] = best[(i, j)] if (i, j) in best else s"),
    "roles not exchanged": ("for d in (2 * p + 1, 2 * p):", "for d in (2 * p, 2 * p + 1):"),
    "true positive with swapped indices": ("if int(truth[s0 + i]) == j)", "if int(truth[s0 + j]) == i)"),
    "known pairs counted over target sentences": ("range(int(do[2 * p]), int(do[2 * p + 1])) if int(truth[i]) >= 0",
                                                  "range(int(do[2 * p]), int(do[2 * p + 2])) if int(truth[i]) >= 0"),
    "ties go to the last setting": ("if f1[k] > f1[best]:", "if f1[k] >= f1[best]:"),
    "precision instead of F1": ("Fraction(2 * t, s + n_truth) if s + n_truth > 0",
                                "Fraction(t, s) if s > 0"),
}


def _run_py_pins(m):
    failed = []
    for c in (check_bidi_hand_examples, check_bidi_identities, check_bidi_special_cases,
              check_bidi_exact_inverse_transposes, check_f1_hand_example, check_f1_closed_forms):
        try:
            c(m)
        except (AssertionError, ZeroDivisionError, IndexError, KeyError):
            failed.append(c)
    return failed


@pytest.mark.parametrize("name", sorted(_PY_MUTANTS))
def test_planted_mistake_in_union_or_objective_is_caught(name, tmp_path):
    import importlib.util
    old, new = _PY_MUTANTS[name]
    src = open(O.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique in the oracle"
    path = tmp_path / "oracle_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_mutant", str(path))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m._lib = O.lib()   # the unmutated C part
    assert _run_py_pins(m), f"no pin caught the planted mistake {name!r}"


def test_unmutated_union_and_objective_pass_all_pins():
    assert _run_py_pins(O) == []


# ------------------------------- contrast without the path constraint (Section 4)

def check_best_match_hand_example(m=O):
    g = _gold("best_match_hand_example.json")
    sel, rep = m.best_match(np.asarray(g["M"], np.int32), g["theta"])
    assert [list(t) for t in sel] == g["selected"] and rep == g["repeated"]


def test_best_match_hand_example():
    check_best_match_hand_example()


def check_best_match_closed_forms(m=O):
    # a permutation matrix of high scores: every row takes its own column, no repeats
    perm = np.random.default_rng(3).permutation(9)
    M = np.full((9, 9), 1000, np.int32)
    M[np.arange(9), perm] = 60000
    sel, rep = m.best_match(M, 32768)
    assert sel == [(i, int(perm[i]), 60000) for i in range(9)] and rep == 0
    # one dominant column: every row takes it, one repeated target
    M = np.full((5, 4), 1000, np.int32)
    M[:, 2] = 50000
    sel, rep = m.best_match(M, 32768)
    assert [j for _, j, _ in sel] == [2] * 5 and rep == 1
    # a constant matrix takes column 0 (lowest index among equals); the
    # threshold is strict
    M = np.full((3, 6), 40000, np.int32)
    assert m.best_match(M, 39999)[0] == [(i, 0, 40000) for i in range(3)]
    assert m.best_match(M, 40000) == ([], 0)
    # no target sentences, no source sentences
    assert m.best_match(np.zeros((4, 0), np.int32), 0) == ([], 0)
    assert m.best_match(np.zeros((0, 4), np.int32), 0) == ([], 0)
    # every source sentence the monotone alignment keeps has a cell above the
    # threshold, so the best match keeps it too (with its row maximum)
    rng = np.random.default_rng(11)
    for _ in range(20):
        M = synth.random_matrix(rng, int(rng.integers(1, 12)), int(rng.integers(1, 12)), lo=0, hi=65536)
        nw = O.align(M, [(-65536, 32768)])[0][1]
        bm, _ = m.best_match(M, 32768)
        assert {i for i, _, _ in nw} <= {i for i, _, _ in bm}
        for i, j, s in bm:
            assert s == M[i].max() and M[i, :j].max(initial=-1) < s


def test_best_match_closed_forms():
    check_best_match_closed_forms()


_BM_MUTANTS = {
    "ties to the last column": ("            if row[c] > row[j]:\n                j = c", "            if row[c] >= row[j]:\n                j = c"),
    "threshold not strict": ("        if row[j] > theta:\n            sel.append", "        if row[j] >= theta:\n            sel.append"),
    "repeats counted per occurrence": ("return sel, sum(1 for c in taken.values() if c > 1)",
                                       "return sel, sum(c for c in taken.values() if c > 1)"),
}


@pytest.mark.parametrize("name", sorted(_BM_MUTANTS))
def test_planted_mistake_in_best_match_is_caught(name, tmp_path):
    import importlib.util
    old, new = _BM_MUTANTS[name]
    src = open(O.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique in the oracle"
    path = tmp_path / "oracle_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_mutant", str(path))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m._lib = O.lib()
    failed = []
    for c in (check_best_match_hand_example, check_best_match_closed_forms):
        try:
            c(m)
        except AssertionError:
            failed.append(c)
    assert failed, f"no pin caught the planted mistake {name!r}"
