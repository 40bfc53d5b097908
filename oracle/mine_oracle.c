/*
 * mine_oracle.c -- plain, slow, obviously-correct CPU oracle of the mining path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it follows (Wolk & Marasek, "Tuned and GPU-accelerated parallel data
 * mining from comparable corpora"):
 *   - Section 4: the comparison of the two sentence sequences of an article pair
 *     is a Needleman-Wunsch global alignment over the sentence-pair matrix M; a
 *     path may not go upward or leftward, i.e. it is monotone and each sentence
 *     is used at most once.
 *   - Section 4: "Penalty" controls how much skipping ahead is allowed -> the
 *     gap score g (<= 0) paid for every unmatched sentence.
 *   - Section 4: "Threshold" accepts an aligned pair as good when its confidence
 *     passes it -> keep matched pairs whose score is strictly above theta.
 * The paper's confidence is an SVM probability whose weights are not available;
 * it is replaced by the fixed-point token-overlap + length score below.  The
 * paper fixes neither the score, the recurrence details, the tie-break nor the
 * rounding; the readings taken here are:
 *   score   s = (W_OV*((q_t+q_s)>>1) + W_LEN*q_l) >> 16, W_OV=49152, W_LEN=16384
 *           q_t = a*65536 / m_j,  a = |U_i intersect V_j|   (0 if m_j = 0)
 *           q_s = b*65536 / n_i,  b = #{t in X_i : dict(t) meets V_j} (0 if n_i = 0)
 *           q_l = min(L,L')*65536 / max(L,L')   (65536 if both are empty)
 *           X_i distinct source tokens, n_i = |X_i|, L = token count,
 *           U_i = distinct union of dict(t), t in X_i (unknown tokens add none),
 *           V_j distinct target tokens, m_j = |V_j|, L' = token count;
 *           all divisions floor divisions of non-negative integers.
 *   NW      H[0][0]=0, H[i][0]=i*g, H[0][j]=j*g,
 *           H[i][j] = max(H[i-1][j-1]+s(i,j), H[i-1][j]+g, H[i][j-1]+g),
 *           direction DIAG if the diagonal attains the max, else UP, else LEFT
 *           (first row LEFT, first column UP).
 *   real    the same features with exact division, in double:
 *           s = 0.75 * (a/m_j + b/n_i) / 2 + 0.25 * min(L,L')/max(L,L')
 *           (a/m_j = 0 if m_j = 0, b/n_i = 0 if n_i = 0, ratio 1 if both are
 *           empty) -- the reference of the single-precision score variant;
 *           65536*s exceeds the fixed-point s by less than 2.375.
 *   path    from (S,T) follow the directions back to (0,0).
 *   select  every DIAG step (i,j) with s(i,j) > theta, in increasing i.
 * Arithmetic is int64 throughout, so nothing here can overflow for inputs the
 * library accepts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_DIAG = 0, OR_UP = 1, OR_LEFT = 2 };

/* ------------------------------------------------------------------ dictionary
 * A sorted copy of the keys; lookup by bisection.  Deliberately unlike any
 * hash table. */
typedef struct {
    int32_t n;
    int32_t *key;     /* sorted */
    int32_t *off;     /* translations of key[k]: tr[off[k] .. off[k]+cnt[k]) */
    int32_t *cnt;
    int32_t *tr;
} oracle_dict;

static const int32_t *g_sort_keys;
static int cmp_by_key(const void *a, const void *b)
{
    int32_t x = g_sort_keys[*(const int32_t *)a], y = g_sort_keys[*(const int32_t *)b];
    return (x > y) - (x < y);
}

void *oracle_dict_new(const int32_t *keys, const int32_t *trans_off, const int32_t *trans,
                      int32_t n_keys)
{
    oracle_dict *d = (oracle_dict *)calloc(1, sizeof(oracle_dict));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_keys > 0 ? n_keys : 1));
    for (int32_t k = 0; k < n_keys; ++k) perm[k] = k;
    g_sort_keys = keys;
    qsort(perm, (size_t)n_keys, sizeof(int32_t), cmp_by_key);
    d->n = n_keys;
    d->key = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_keys > 0 ? n_keys : 1));
    d->off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_keys > 0 ? n_keys : 1));
    d->cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_keys > 0 ? n_keys : 1));
    int64_t total = n_keys > 0 ? trans_off[n_keys] : 0;
    d->tr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (total > 0) memcpy(d->tr, trans, sizeof(int32_t) * (size_t)total);
    for (int32_t k = 0; k < n_keys; ++k) {
        int32_t o = perm[k];
        d->key[k] = keys[o];
        d->off[k] = trans_off[o];
        d->cnt[k] = trans_off[o + 1] - trans_off[o];
    }
    free(perm);
    return d;
}

void oracle_dict_free(void *h)
{
    oracle_dict *d = (oracle_dict *)h;
    if (!d) return;
    free(d->key); free(d->off); free(d->cnt); free(d->tr); free(d);
}

/* translations of token t: returns count, *out points into the table */
static int32_t dict_lookup(const oracle_dict *d, int32_t t, const int32_t **out)
{
    int32_t lo = 0, hi = d->n - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (d->key[mid] == t) { *out = d->tr + d->off[mid]; return d->cnt[mid]; }
        if (d->key[mid] < t) lo = mid + 1; else hi = mid - 1;
    }
    *out = NULL;
    return 0;
}

/* ------------------------------------------------------------------ sets */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sort v[0..n) and drop repeats; returns the distinct count */
static int32_t sort_unique(int32_t *v, int32_t n)
{
    if (n <= 1) return n;
    qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
    int32_t w = 1;
    for (int32_t r = 1; r < n; ++r)
        if (v[r] != v[w - 1]) v[w++] = v[r];
    return w;
}

static int contains(const int32_t *sorted, int32_t n, int32_t x)
{
    int32_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (sorted[mid] == x) return 1;
        if (sorted[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

typedef struct {
    int32_t *X; int32_t n;   /* distinct source tokens (sorted) */
    int32_t *U; int32_t nu;  /* distinct translations (sorted) */
    int64_t L;               /* token count */
} src_set;

typedef struct {
    int32_t *V; int32_t m;   /* distinct target tokens (sorted) */
    int64_t L;
} tgt_set;

/* ------------------------------------------------------------------ score
 * Fills M (S x T, row-major, int32) with the fixed-point pair score when M is
 * not NULL, and Mr (double) with the real-valued score when Mr is not NULL. */
static void score_matrix_impl(void *dict, const int32_t *src_off, const int32_t *src_tok, int32_t S,
                              const int32_t *tgt_off, const int32_t *tgt_tok, int32_t T, int32_t *M,
                              double *Mr)
{
    const oracle_dict *d = (const oracle_dict *)dict;
    src_set *src = (src_set *)calloc((size_t)(S > 0 ? S : 1), sizeof(src_set));
    tgt_set *tgt = (tgt_set *)calloc((size_t)(T > 0 ? T : 1), sizeof(tgt_set));

    for (int32_t i = 0; i < S; ++i) {
        int32_t L = src_off[i + 1] - src_off[i];
        src[i].L = L;
        src[i].X = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
        memcpy(src[i].X, src_tok + src_off[i], sizeof(int32_t) * (size_t)L);
        src[i].n = sort_unique(src[i].X, L);
        int64_t cap = 0;
        for (int32_t p = 0; p < src[i].n; ++p) {
            const int32_t *tr;
            cap += dict_lookup(d, src[i].X[p], &tr);
        }
        src[i].U = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
        int32_t w = 0;
        for (int32_t p = 0; p < src[i].n; ++p) {
            const int32_t *tr;
            int32_t c = dict_lookup(d, src[i].X[p], &tr);
            for (int32_t k = 0; k < c; ++k) src[i].U[w++] = tr[k];
        }
        src[i].nu = sort_unique(src[i].U, w);
    }
    for (int32_t j = 0; j < T; ++j) {
        int32_t L = tgt_off[j + 1] - tgt_off[j];
        tgt[j].L = L;
        tgt[j].V = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
        memcpy(tgt[j].V, tgt_tok + tgt_off[j], sizeof(int32_t) * (size_t)L);
        tgt[j].m = sort_unique(tgt[j].V, L);
    }

    for (int32_t i = 0; i < S; ++i) {
        for (int32_t j = 0; j < T; ++j) {
            /* a = |U_i intersect V_j| by merging two sorted distinct lists */
            int64_t a = 0;
            int32_t x = 0, y = 0;
            while (x < src[i].nu && y < tgt[j].m) {
                if (src[i].U[x] == tgt[j].V[y]) { ++a; ++x; ++y; }
                else if (src[i].U[x] < tgt[j].V[y]) ++x;
                else ++y;
            }
            /* b = number of distinct source tokens with a translation in V_j */
            int64_t b = 0;
            for (int32_t p = 0; p < src[i].n; ++p) {
                const int32_t *tr;
                int32_t c = dict_lookup(d, src[i].X[p], &tr);
                int hit = 0;
                for (int32_t k = 0; k < c && !hit; ++k) hit = contains(tgt[j].V, tgt[j].m, tr[k]);
                b += hit;
            }
            int64_t q_t = tgt[j].m > 0 ? (a * 65536) / tgt[j].m : 0;
            int64_t q_s = src[i].n > 0 ? (b * 65536) / src[i].n : 0;
            int64_t lmin = src[i].L < tgt[j].L ? src[i].L : tgt[j].L;
            int64_t lmax = src[i].L < tgt[j].L ? tgt[j].L : src[i].L;
            int64_t q_l = lmax > 0 ? (lmin * 65536) / lmax : 65536;
            int64_t s = (49152 * ((q_t + q_s) / 2) + 16384 * q_l) / 65536;
            if (M) M[(int64_t)i * T + j] = (int32_t)s;
            if (Mr) {
                double rt = tgt[j].m > 0 ? (double)a / (double)tgt[j].m : 0.0;
                double rs = src[i].n > 0 ? (double)b / (double)src[i].n : 0.0;
                double rl = lmax > 0 ? (double)lmin / (double)lmax : 1.0;
                Mr[(int64_t)i * T + j] = 0.75 * (rt + rs) / 2.0 + 0.25 * rl;
            }
        }
    }
    for (int32_t i = 0; i < S; ++i) { free(src[i].X); free(src[i].U); }
    for (int32_t j = 0; j < T; ++j) free(tgt[j].V);
    free(src); free(tgt);
}

void oracle_score_matrix(void *dict, const int32_t *src_off, const int32_t *src_tok, int32_t S,
                         const int32_t *tgt_off, const int32_t *tgt_tok, int32_t T, int32_t *M)
{
    score_matrix_impl(dict, src_off, src_tok, S, tgt_off, tgt_tok, T, M, NULL);
}

void oracle_score_matrix_f64(void *dict, const int32_t *src_off, const int32_t *src_tok, int32_t S,
                             const int32_t *tgt_off, const int32_t *tgt_tok, int32_t T, double *Mr)
{
    score_matrix_impl(dict, src_off, src_tok, S, tgt_off, tgt_tok, T, NULL, Mr);
}

/* ------------------------------------------------------------------ NW
 * H: (S+1)*(T+1) int64 (may be NULL: then a private one is used),
 * D: (S+1)*(T+1) uint8 directions.  Returns H[S][T]. */
int64_t oracle_nw(const int32_t *M, int32_t S, int32_t T, int32_t g, int64_t *H, uint8_t *D)
{
    const int64_t W = (int64_t)T + 1;
    int64_t *h = H ? H : (int64_t *)malloc(sizeof(int64_t) * (size_t)((S + 1) * W));
    h[0] = 0;
    D[0] = OR_DIAG; /* unused corner */
    for (int32_t j = 1; j <= T; ++j) { h[j] = (int64_t)j * g; D[j] = OR_LEFT; }
    for (int32_t i = 1; i <= S; ++i) {
        h[i * W] = (int64_t)i * g;
        D[i * W] = OR_UP;
        for (int32_t j = 1; j <= T; ++j) {
            int64_t diag = h[(i - 1) * W + (j - 1)] + M[(int64_t)(i - 1) * T + (j - 1)];
            int64_t up = h[(i - 1) * W + j] + g;
            int64_t left = h[i * W + (j - 1)] + g;
            int64_t best = diag;
            if (up > best) best = up;
            if (left > best) best = left;
            h[i * W + j] = best;
            D[i * W + j] = (diag == best) ? OR_DIAG : (up == best) ? OR_UP : OR_LEFT;
        }
    }
    int64_t r = h[S * W + T];
    if (!H) free(h);
    return r;
}

/* Walk the directions from (S,T) to (0,0).  moves[k] (k = 0 is the LAST
 * move of the path, i.e. the one entering (S,T)).  Returns the move count. */
int32_t oracle_traceback(const uint8_t *D, int32_t S, int32_t T, uint8_t *moves)
{
    const int64_t W = (int64_t)T + 1;
    int32_t i = S, j = T, k = 0;
    while (i > 0 || j > 0) {
        uint8_t m = D[i * W + j];
        moves[k++] = m;
        if (m == OR_DIAG) { --i; --j; }
        else if (m == OR_UP) --i;
        else --j;
    }
    return k;
}

/* Matched pairs of a path with s > theta, in increasing i; 0-based indices.
 * out: 3 int32 per pair (i, j, s).  Returns the count. */
int32_t oracle_select(const int32_t *M, int32_t S, int32_t T, const uint8_t *moves, int32_t n_moves,
                      int32_t theta, int32_t *out)
{
    /* replay the path forward from (0,0) so pairs come out in increasing i */
    int32_t i = 0, j = 0, n = 0;
    (void)S;
    for (int32_t k = n_moves - 1; k >= 0; --k) {
        uint8_t m = moves[k];
        if (m == OR_DIAG) {
            ++i; ++j;
            int32_t s = M[(int64_t)(i - 1) * T + (j - 1)];
            if (s > theta) { out[3 * n] = i - 1; out[3 * n + 1] = j - 1; out[3 * n + 2] = s; ++n; }
        } else if (m == OR_UP) ++i;
        else ++j;
    }
    return n;
}

/* NW + traceback + select on a given matrix, for n_set (gap, theta) settings.
 * nw_score[n_set]; sel_cnt[n_set]; sel: n_set blocks of min(S,T) triples. */
void oracle_align(const int32_t *M, int32_t S, int32_t T, int32_t n_set, const int32_t *gaps,
                  const int32_t *thetas, int64_t *nw_score, int32_t *sel_cnt, int32_t *sel)
{
    size_t cells = (size_t)(S + 1) * (size_t)(T + 1);
    uint8_t *D = (uint8_t *)malloc(cells);
    uint8_t *moves = (uint8_t *)malloc((size_t)S + (size_t)T + 1);
    int32_t cap = S < T ? S : T;
    for (int32_t k = 0; k < n_set; ++k) {
        nw_score[k] = oracle_nw(M, S, T, gaps[k], NULL, D);
        int32_t nm = oracle_traceback(D, S, T, moves);
        sel_cnt[k] = oracle_select(M, S, T, moves, nm, thetas[k], sel + (size_t)3 * cap * k);
    }
    free(D);
    free(moves);
}

/* Whole path for a packed batch (see the synthetic generator for the layout):
 * pairs are independent, so they are spread over OpenMP threads when the
 * library was built with OpenMP.  For pair p and setting k:
 *   nw_score[p*n_set+k], sel_cnt[p*n_set+k],
 *   sel + 3*(sel_base[p]*n_set + k*min(S_p,T_p))   (caller sizes sel_base). */
int32_t oracle_mine_batch(void *dict, int32_t P, const int32_t *doc_off, const int32_t *sent_off,
                          const int32_t *tokens, int32_t n_set, const int32_t *gaps,
                          const int32_t *thetas, const int64_t *sel_base, int64_t *nw_score,
                          int32_t *sel_cnt, int32_t *sel, int32_t n_threads)
{
    int32_t used = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t p = 0; p < P; ++p) {
        int32_t s0 = doc_off[2 * p], s1 = doc_off[2 * p + 1], s2 = doc_off[2 * p + 2];
        int32_t S = s1 - s0, T = s2 - s1;
        int32_t *so = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S + 1));
        int32_t *to = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
        for (int32_t i = 0; i <= S; ++i) so[i] = sent_off[s0 + i] - sent_off[s0];
        for (int32_t j = 0; j <= T; ++j) to[j] = sent_off[s1 + j] - sent_off[s1];
        int32_t *M = (int32_t *)malloc(sizeof(int32_t) * (size_t)((int64_t)S * T > 0 ? (int64_t)S * T : 1));
        oracle_score_matrix(dict, so, tokens + sent_off[s0], S, to, tokens + sent_off[s1], T, M);
        oracle_align(M, S, T, n_set, gaps, thetas, nw_score + (int64_t)p * n_set,
                     sel_cnt + (int64_t)p * n_set, sel + (int64_t)3 * sel_base[p] * n_set);
        free(M); free(so); free(to);
    }
    (void)n_threads;
    return used;
}
