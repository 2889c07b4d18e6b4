/*
 * CPU oracle for the exhaustive epistasis search of Fiuncho
 * (Ponte-Fernandez, Gonzalez-Dominguez, Martin: "Fiuncho: a program for
 * any-order epistasis detection in CPU clusters").
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plainly correct statement of
 * what the GPU search computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it; the library
 * never does, and the two share no code, header or table.
 *
 * What it computes, in the paper's terms:
 *   - genotype values 0/1/2 per SNP (rows a_1, a_2, a_3 of a genotype table,
 *     Section "Constructing the genotype tables", Fig. 2);
 *   - the 3^k x {cases, controls} contingency table of a k-combination,
 *     counted sample by sample with no bit vectors (Section "Computing the
 *     contingency tables", Fig. 3).  Cell order is first-SNP-major
 *     (a1b1, a1b2, ..., a3b3), column 0 = cases;
 *   - mutual information MI = H(X) + H(Y) - H(X,Y) with plug-in entropies
 *     H = -sum p ln p over nonzero cells, natural log, FP64 (Section "Mutual
 *     Information test", the MI and entropy equations);
 *   - the exhaustive search of Algorithm 1: (k-1)-prefixes in ascending
 *     lexicographic order are dealt round-robin to threads (Section
 *     "Distribution strategy", Fig. 4); each thread keeps an ascending
 *     sorted list of the best combinations with the sorted_insert rule;
 *     the per-thread lists are joined, sorted and truncated (end of Section
 *     "Algorithmic implementation").
 *
 * Readings where the paper is silent or garbled:
 *   - extension SNPs run over j = i_{k-1}+1 .. n-1 (0-based): combinations
 *     without repetition;
 *   - ties are broken by the lexicographic order of the index tuple: of two
 *     equal scores the smaller tuple ranks first (the single-thread
 *     sorted_insert keeps the earlier-enumerated one);
 *   - phenotype 1 = case, 0 = control; log base e.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_KMAX 10

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ERANGE = -2, ORC_ENOMEM = -3 };

static int64_t ipow3(int k)
{
    int64_t r = 1;
    for (int i = 0; i < k; ++i) r *= 3;
    return r;
}

/* Binomial coefficient C(n, r) in exact 128-bit arithmetic; saturates at
 * INT64_MAX (reported as too large by the callers). */
int64_t orc_binom(int64_t n, int64_t r)
{
    if (r < 0 || n < 0 || r > n) return 0;
    if (r > n - r) r = n - r;
    unsigned __int128 acc = 1;
    for (int64_t i = 1; i <= r; ++i) {
        acc = acc * (unsigned __int128)(n - r + i) / (unsigned __int128)i;
        if (acc > (unsigned __int128)INT64_MAX) return INT64_MAX;
    }
    return (int64_t)acc;
}

int orc_validate(const uint8_t *G, int64_t S, int64_t M, const uint8_t *ph, int k)
{
    if (!G || !ph || S <= 0 || M <= 0) return ORC_EINVAL;
    if (k < 1 || k > ORC_KMAX || k > S) return ORC_EINVAL;
    for (int64_t i = 0; i < S * M; ++i)
        if (G[i] > 2) return ORC_EINVAL;
    for (int64_t m = 0; m < M; ++m)
        if (ph[m] > 1) return ORC_EINVAL;
    return ORC_OK;
}

/* Contingency table of one k-combination, counted one sample at a time.
 * T is [3^k][2]: T[cell][0] = cases, T[cell][1] = controls, where
 * cell = sum_t g[combo[t]][m] * 3^(k-1-t). */
void orc_table_one(const uint8_t *G, int64_t M, const uint8_t *ph, int k,
                   const uint32_t *combo, uint32_t *T)
{
    const int64_t cells = ipow3(k);
    memset(T, 0, sizeof(uint32_t) * (size_t)(2 * cells));
    for (int64_t m = 0; m < M; ++m) {
        int64_t cell = 0;
        for (int t = 0; t < k; ++t)
            cell = cell * 3 + G[(int64_t)combo[t] * M + m];
        int col = ph[m] == 1 ? 0 : 1;
        T[cell * 2 + col] += 1;
    }
}

/* MI(X;Y) = H(X) + H(Y) - H(X,Y) from a [cells][2] count table, p = n/N. */
double orc_mi_table(const uint32_t *T, int64_t cells)
{
    double N = 0.0, ny0 = 0.0, ny1 = 0.0;
    for (int64_t x = 0; x < cells; ++x) {
        ny0 += (double)T[2 * x];
        ny1 += (double)T[2 * x + 1];
    }
    N = ny0 + ny1;
    if (N <= 0.0) return 0.0;
    double hx = 0.0, hxy = 0.0, hy = 0.0;
    for (int64_t x = 0; x < cells; ++x) {
        double nx = (double)T[2 * x] + (double)T[2 * x + 1];
        if (nx > 0.0) hx -= (nx / N) * log(nx / N);
        for (int y = 0; y < 2; ++y) {
            double nxy = (double)T[2 * x + y];
            if (nxy > 0.0) hxy -= (nxy / N) * log(nxy / N);
        }
    }
    if (ny0 > 0.0) hy -= (ny0 / N) * log(ny0 / N);
    if (ny1 > 0.0) hy -= (ny1 / N) * log(ny1 / N);
    return hx + hy - hxy;
}

/* Tables of n caller-given combinations: out is [n][3^k][2]. */
int orc_tables(const uint8_t *G, int64_t S, int64_t M, const uint8_t *ph, int k,
               const uint32_t *combos, int64_t n, uint32_t *out)
{
    if (!G || !ph || !combos || !out || k < 1 || k > ORC_KMAX || n < 0) return ORC_EINVAL;
    const int64_t cells = ipow3(k);
    for (int64_t c = 0; c < n; ++c) {
        for (int t = 0; t < k; ++t)
            if ((int64_t)combos[c * k + t] >= S) return ORC_ERANGE;
        orc_table_one(G, M, ph, k, combos + c * k, out + c * cells * 2);
    }
    return ORC_OK;
}

/* MI of n tables laid out [n][cells][2]. */
int orc_mi(const uint32_t *tables, int64_t n, int k, double *out)
{
    if (!tables || !out || k < 1 || k > ORC_KMAX) return ORC_EINVAL;
    const int64_t cells = ipow3(k);
    for (int64_t c = 0; c < n; ++c) out[c] = orc_mi_table(tables + c * cells * 2, cells);
    return ORC_OK;
}

/* ----- search (Algorithm 1) ------------------------------------------ */

typedef struct {
    double score;
    uint32_t idx[ORC_KMAX];
} orc_entry;

/* Strict ranking: a ranks above b if its score is larger, or the scores are
 * equal and its index tuple is lexicographically smaller. */
static int ranks_above(const orc_entry *a, const orc_entry *b, int k)
{
    if (a->score != b->score) return a->score > b->score;
    for (int t = 0; t < k; ++t)
        if (a->idx[t] != b->idx[t]) return a->idx[t] < b->idx[t];
    return 0;
}

typedef struct {
    orc_entry *list; /* ascending: list[0] is the weakest kept entry */
    int64_t size, cap;
    int k;
} orc_list;

/* sorted_insert of Algorithm 1 with the full ranking key. */
static void sorted_insert(orc_list *L, const orc_entry *e)
{
    if (L->cap <= 0) return;
    if (L->size < L->cap || ranks_above(e, &L->list[0], L->k)) {
        int64_t i = 0;
        while (i < L->size && !ranks_above(&L->list[i], e, L->k)) ++i;
        memmove(&L->list[i + 1], &L->list[i], sizeof(orc_entry) * (size_t)(L->size - i));
        L->list[i] = *e;
        L->size += 1;
        if (L->size > L->cap) {
            memmove(&L->list[0], &L->list[1], sizeof(orc_entry) * (size_t)(L->size - 1));
            L->size -= 1;
        }
    }
}

/* Advance a (k-1)-prefix over [0, n-2] in lexicographic order; the last
 * element stops at n-2 so that every prefix has at least one extension.
 * Returns 0 when exhausted. */
static int next_prefix(uint32_t *p, int len, int64_t n)
{
    if (len == 0) return 0;
    int t = len - 1;
    while (t >= 0 && (int64_t)p[t] == n - 1 - (len - t)) --t;
    if (t < 0) return 0;
    p[t] += 1;
    for (int u = t + 1; u < len; ++u) p[u] = p[u - 1] + 1;
    return 1;
}

typedef struct {
    const uint8_t *G, *ph;
    int64_t S, M;
    int k, unit, units;
    int64_t pfx_begin, pfx_end; /* prefix ordinals handled by the search */
    orc_list list;
    int64_t tested;
    uint64_t *count_only; /* distribution mode: count combinations only */
} orc_task;

static void *search_unit(void *arg)
{
    orc_task *w = (orc_task *)arg;
    const int k = w->k;
    const int plen = k - 1;
    const int64_t cells = ipow3(k);
    uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * cells));
    uint32_t pfx[ORC_KMAX];
    for (int t = 0; t < plen; ++t) pfx[t] = (uint32_t)t;
    int64_t ordinal = 0;
    int more = (plen == 0) ? 1 : ((int64_t)plen <= w->S - 1);
    while (more) {
        if (ordinal >= w->pfx_end) break;
        if (ordinal >= w->pfx_begin && (ordinal % w->units) == w->unit) {
            orc_entry e;
            for (int t = 0; t < plen; ++t) e.idx[t] = pfx[t];
            int64_t j0 = plen == 0 ? 0 : (int64_t)pfx[plen - 1] + 1;
            for (int64_t j = j0; j < w->S; ++j) {
                w->tested += 1;
                if (w->count_only) { w->count_only[w->unit] += 1; continue; }
                e.idx[plen] = (uint32_t)j;
                orc_table_one(w->G, w->M, w->ph, k, e.idx, T);
                e.score = orc_mi_table(T, cells);
                sorted_insert(&w->list, &e);
            }
        }
        ordinal += 1;
        more = next_prefix(pfx, plen, w->S);
    }
    free(T);
    return NULL;
}

static int cmp_desc(const void *a, const void *b, void *kp)
{
    int k = *(int *)kp;
    const orc_entry *x = (const orc_entry *)a, *y = (const orc_entry *)b;
    if (ranks_above(x, y, k)) return -1;
    if (ranks_above(y, x, k)) return 1;
    return 0;
}

static int resolve_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/*
 * Exhaustive search over the (k-1)-prefix ordinals [pfx_begin, pfx_end)
 * (pfx_end < 0 means all C(S-1, k-1) prefixes).  Writes the best
 * min(top_n, tested) combinations, best first, to out_idx [count][k] and
 * out_score [count]; *out_count gets that count, *out_tested the number of
 * combinations scored.
 */
int orc_search(const uint8_t *G, int64_t S, int64_t M, const uint8_t *ph, int k,
               int64_t top_n, int nthreads, int64_t pfx_begin, int64_t pfx_end,
               uint32_t *out_idx, double *out_score, int64_t *out_count,
               int64_t *out_tested)
{
    int rc = orc_validate(G, S, M, ph, k);
    if (rc) return rc;
    if (top_n < 0 || !out_count) return ORC_EINVAL;
    if (top_n > 0 && (!out_idx || !out_score)) return ORC_EINVAL;
    const int64_t nprefix = k == 1 ? 1 : orc_binom(S - 1, k - 1);
    if (pfx_end < 0 || pfx_end > nprefix) pfx_end = nprefix;
    if (pfx_begin < 0) pfx_begin = 0;
    int units = resolve_threads(nthreads);
    orc_task *w = (orc_task *)calloc((size_t)units, sizeof(orc_task));
    pthread_t *th = (pthread_t *)calloc((size_t)units, sizeof(pthread_t));
    if (!w || !th) { free(w); free(th); return ORC_ENOMEM; }
    for (int u = 0; u < units; ++u) {
        w[u] = (orc_task){.G = G, .ph = ph, .S = S, .M = M, .k = k, .unit = u,
                          .units = units, .pfx_begin = pfx_begin, .pfx_end = pfx_end};
        w[u].list.k = k;
        w[u].list.cap = top_n;
        w[u].list.list = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(top_n + 1));
        if (!w[u].list.list) {
            for (int v = 0; v <= u; ++v) free(w[v].list.list);
            free(w);
            free(th);
            return ORC_ENOMEM;
        }
    }
    for (int u = 0; u < units; ++u) pthread_create(&th[u], NULL, search_unit, &w[u]);
    int64_t total = 0, tested = 0;
    for (int u = 0; u < units; ++u) {
        pthread_join(th[u], NULL);
        total += w[u].list.size;
        tested += w[u].tested;
    }
    /* Join the per-thread lists, sort best first and truncate. */
    orc_entry *all = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(total + 1));
    int64_t n = 0;
    for (int u = 0; u < units; ++u) {
        memcpy(all + n, w[u].list.list, sizeof(orc_entry) * (size_t)w[u].list.size);
        n += w[u].list.size;
        free(w[u].list.list);
    }
    qsort_r(all, (size_t)n, sizeof(orc_entry), cmp_desc, &k);
    int64_t cnt = n < top_n ? n : top_n;
    for (int64_t i = 0; i < cnt; ++i) {
        for (int t = 0; t < k; ++t) out_idx[i * k + t] = all[i].idx[t];
        out_score[i] = all[i].score;
    }
    *out_count = cnt;
    if (out_tested) *out_tested = tested;
    free(all);
    free(w);
    free(th);
    return ORC_OK;
}

/*
 * The static distribution of Section "Distribution strategy" (Fig. 4):
 * combinations assigned to each of p units when the (k-1)-prefixes with at
 * least one extension are dealt round-robin in ascending order.
 * counts has p entries.
 */
int orc_distribution(int64_t n, int k, int p, uint64_t *counts)
{
    /* Section "Distribution strategy" (Fig. 4): the (k-1)-prefixes that have
     * at least one extension are dealt round-robin in ascending lexicographic
     * order; a prefix ending in SNP i brings its n - 1 - i extensions to its
     * unit.  One pass over the prefixes. */
    if (n < 1 || k < 2 || k > ORC_KMAX || k > n || p < 1 || !counts) return ORC_EINVAL;
    memset(counts, 0, sizeof(uint64_t) * (size_t)p);
    const int plen = k - 1;
    uint32_t pfx[ORC_KMAX];
    for (int t = 0; t < plen; ++t) pfx[t] = (uint32_t)t;
    int64_t ordinal = 0;
    int more = (int64_t)plen <= n - 1;
    while (more) {
        counts[ordinal % p] += (uint64_t)(n - 1 - (int64_t)pfx[plen - 1]);
        ordinal += 1;
        more = next_prefix(pfx, plen, n);
    }
    return ORC_OK;
}
