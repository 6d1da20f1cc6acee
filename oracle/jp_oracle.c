/*
 * CPU oracle for the join-project queries -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and
 * its --impl reference arm) may load this library.  The product path never
 * calls it and shares no code with it.
 *
 * What it computes is the plain definition of the queries (Section 2.1):
 *
 *   two-path  Q(x,z)          = { (a,c)      : exists b, (a,b) in R and (c,b) in S }
 *   star      Q*_k(x1..xk)    = { (a1..ak)   : exists b, (ai,b) in Ri for every i }
 *
 * with set semantics (SELECT DISTINCT, Section 1, Example 1).  The paper's
 * Algorithm 1 reaches exactly this set for any thresholds (the correctness
 * argument after Algorithm 1), so the oracle is that definition written out:
 *
 *   1. sort a copy of S (resp. R2..Rk) by y, so the tuples with one y value
 *      form a contiguous run (a sort-based hash join on y);
 *   2. for every R tuple (a,b) whose x lies in the requested value range, find
 *      the run of b in S by binary search and emit (a,c) for every c in it
 *      (for the star, every combination of the k-1 runs);
 *   3. sort the emitted tuples lexicographically (signed int32) and drop
 *      repeats; optionally keep how many witnesses each tuple had.
 *
 * Inputs are SoA int32 arrays and may hold duplicate tuples; duplicates are
 * removed first because relations are sets.  Memory grows with the number of
 * emitted candidates, so callers bound it with the x value range.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t k0, k1; } pair32;

static int cmp_pair(const void* a, const void* b) {
    const pair32* p = (const pair32*)a;
    const pair32* q = (const pair32*)b;
    if (p->k0 != q->k0) return p->k0 < q->k0 ? -1 : 1;
    if (p->k1 != q->k1) return p->k1 < q->k1 ? -1 : 1;
    return 0;
}

/* Distinct (v, y) tuples of one relation, sorted by (y, v). */
static pair32* sorted_by_y(const int32_t* v, const int32_t* y, int64_t n, int64_t* n_out) {
    pair32* t = (pair32*)malloc(sizeof(pair32) * (size_t)(n > 0 ? n : 1));
    if (!t) return NULL;
    for (int64_t i = 0; i < n; ++i) { t[i].k0 = y[i]; t[i].k1 = v[i]; }
    qsort(t, (size_t)n, sizeof(pair32), cmp_pair);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || cmp_pair(&t[m - 1], &t[i]) != 0) t[m++] = t[i];
    *n_out = m;
    return t;
}

/* First index i in t[0..n) with t[i].k0 >= key. */
static int64_t lower_y(const pair32* t, int64_t n, int32_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t[mid].k0 < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * Two-path query restricted to R tuples with x in [x_lo, x_hi] (values).
 * Writes up to `cap` distinct sorted pairs to out_x/out_z and, when
 * out_cnt is non-NULL, the number of distinct witnesses b of each pair.
 * Returns the number of distinct pairs (which may exceed cap: call again
 * with a bigger buffer), or -1 when memory runs out.
 */
int64_t oracle_two_path(const int32_t* rx, const int32_t* ry, int64_t nr,
                        const int32_t* sz, const int32_t* sy, int64_t ns,
                        int32_t x_lo, int32_t x_hi,
                        int32_t* out_x, int32_t* out_z, int32_t* out_cnt, int64_t cap) {
    int64_t nsd = 0, nrd = 0;
    pair32* s = sorted_by_y(sz, sy, ns, &nsd);
    pair32* r = sorted_by_y(rx, ry, nr, &nrd);   /* dedup R; (y, x) order */
    if (!s || !r) { free(s); free(r); return -1; }

    /* count candidates to size the buffer */
    int64_t total = 0;
    for (int64_t i = 0; i < nrd; ++i) {
        int32_t a = r[i].k1, b = r[i].k0;
        if (a < x_lo || a > x_hi) continue;
        int64_t lo = lower_y(s, nsd, b);
        int64_t hi = lo;
        while (hi < nsd && s[hi].k0 == b) ++hi;
        total += hi - lo;
    }
    pair32* cand = (pair32*)malloc(sizeof(pair32) * (size_t)(total > 0 ? total : 1));
    if (!cand) { free(s); free(r); return -1; }
    int64_t m = 0;
    for (int64_t i = 0; i < nrd; ++i) {
        int32_t a = r[i].k1, b = r[i].k0;
        if (a < x_lo || a > x_hi) continue;
        for (int64_t j = lower_y(s, nsd, b); j < nsd && s[j].k0 == b; ++j) {
            cand[m].k0 = a;
            cand[m].k1 = s[j].k1;
            ++m;
        }
    }
    qsort(cand, (size_t)m, sizeof(pair32), cmp_pair);
    int64_t d = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && cmp_pair(&cand[i - 1], &cand[i]) == 0) {
            if (out_cnt && d - 1 < cap) out_cnt[d - 1] += 1;
            continue;
        }
        if (d < cap) {
            out_x[d] = cand[i].k0;
            out_z[d] = cand[i].k1;
            if (out_cnt) out_cnt[d] = 1;
        }
        ++d;
    }
    free(cand); free(s); free(r);
    return d;
}

typedef struct { int32_t v[8]; } tup8;
static int g_k = 0;
static int cmp_tup(const void* a, const void* b) {
    const tup8* p = (const tup8*)a;
    const tup8* q = (const tup8*)b;
    for (int i = 0; i < g_k; ++i)
        if (p->v[i] != q->v[i]) return p->v[i] < q->v[i] ? -1 : 1;
    return 0;
}

/*
 * Star query Q*_k (2 <= k <= 8) restricted to R1 tuples with x1 in
 * [x_lo, x_hi].  xs[i], ys[i], ns[i] describe relation R_{i+1}.  Output
 * columns out[i] (each of capacity cap) receive the sorted distinct tuples.
 * Returns the number of distinct tuples, or -1 on failure.
 */
int64_t oracle_star(int k, const int32_t* const* xs, const int32_t* const* ys,
                    const int64_t* ns, int32_t x_lo, int32_t x_hi,
                    int32_t* const* out, int64_t cap) {
    if (k < 2 || k > 8) return -1;
    pair32* rel[8] = {0};
    int64_t nd[8] = {0};
    for (int i = 0; i < k; ++i) {
        rel[i] = sorted_by_y(xs[i], ys[i], ns[i], &nd[i]);
        if (!rel[i]) { for (int j = 0; j < i; ++j) free(rel[j]); return -1; }
    }
    /* pass 1 counts, pass 2 fills */
    tup8* cand = NULL;
    int64_t total = 0, m = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            cand = (tup8*)malloc(sizeof(tup8) * (size_t)(total > 0 ? total : 1));
            if (!cand) { for (int j = 0; j < k; ++j) free(rel[j]); return -1; }
        }
        for (int64_t i = 0; i < nd[0]; ++i) {
            int32_t a1 = rel[0][i].k1, b = rel[0][i].k0;
            if (a1 < x_lo || a1 > x_hi) continue;
            int64_t lo[8], hi[8], cur[8];
            int64_t combos = 1;
            for (int r = 1; r < k; ++r) {
                lo[r] = lower_y(rel[r], nd[r], b);
                hi[r] = lo[r];
                while (hi[r] < nd[r] && rel[r][hi[r]].k0 == b) ++hi[r];
                combos *= (hi[r] - lo[r]);
            }
            if (combos == 0) continue;
            if (pass == 0) { total += combos; continue; }
            for (int r = 1; r < k; ++r) cur[r] = lo[r];
            for (;;) {
                tup8 t;
                memset(&t, 0, sizeof(t));
                t.v[0] = a1;
                for (int r = 1; r < k; ++r) t.v[r] = rel[r][cur[r]].k1;
                cand[m++] = t;
                int r = k - 1;
                while (r >= 1) {
                    if (++cur[r] < hi[r]) break;
                    cur[r] = lo[r];
                    --r;
                }
                if (r < 1) break;
            }
        }
    }
    g_k = k;
    qsort(cand, (size_t)m, sizeof(tup8), cmp_tup);
    int64_t d = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && cmp_tup(&cand[i - 1], &cand[i]) == 0) continue;
        if (d < cap)
            for (int r = 0; r < k; ++r) out[r][d] = cand[i].v[r];
        ++d;
    }
    free(cand);
    for (int j = 0; j < k; ++j) free(rel[j]);
    return d;
}

/*
 * Distinct z values of one x value a in the two-path query, sorted: the
 * per-row form of the definition used to check single rows of very large
 * outputs.  `s_sorted` must hold S as (y, z) pairs sorted and deduplicated
 * (see oracle_sort_by_y).  Returns the number of values (may exceed cap).
 */
int64_t oracle_two_path_row(const int32_t* r_y_of_a, int64_t deg_a,
                            const int32_t* s_y_sorted, const int32_t* s_z_sorted, int64_t ns,
                            int32_t* out_z, int64_t cap) {
    int64_t total = 0;
    for (int64_t i = 0; i < deg_a; ++i) {
        int32_t b = r_y_of_a[i];
        int64_t lo = 0, hi = ns;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (s_y_sorted[mid] < b) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < ns && s_y_sorted[j] == b; ++j) ++total;
    }
    pair32* c = (pair32*)malloc(sizeof(pair32) * (size_t)(total > 0 ? total : 1));
    if (!c) return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < deg_a; ++i) {
        int32_t b = r_y_of_a[i];
        int64_t lo = 0, hi = ns;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (s_y_sorted[mid] < b) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < ns && s_y_sorted[j] == b; ++j) { c[m].k0 = s_z_sorted[j]; c[m].k1 = 0; ++m; }
    }
    qsort(c, (size_t)m, sizeof(pair32), cmp_pair);
    int64_t d = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && c[i - 1].k0 == c[i].k0) continue;
        if (d < cap) out_z[d] = c[i].k0;
        ++d;
    }
    free(c);
    return d;
}

/*
 * The two-path rows of several x values: row i's y values are
 * r_y[r_off[i] .. r_off[i+1]); each row is answered as oracle_two_path_row
 * does (join with S sorted by y, sort, unique) and the rows' distinct z are
 * written one after another (up to cap values in total); out_cnt[i] receives
 * row i's count.  Returns the total number of values (may exceed cap), or -1
 * when memory runs out.
 */
int64_t oracle_two_path_rows(const int64_t* r_off, int64_t nrows, const int32_t* r_y,
                             const int32_t* s_y_sorted, const int32_t* s_z_sorted, int64_t ns,
                             int32_t* out_z, int64_t cap, int64_t* out_cnt) {
    int64_t total = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        int32_t* dst = total < cap ? out_z + total : NULL;
        int64_t room = total < cap ? cap - total : 0;
        int32_t dummy;
        int64_t d = oracle_two_path_row(r_y + r_off[i], r_off[i + 1] - r_off[i], s_y_sorted,
                                        s_z_sorted, ns, dst ? dst : &dummy, room);
        if (d < 0) return -1;
        out_cnt[i] = d;
        total += d;
    }
    return total;
}

/* Sort and deduplicate (y, v) pairs; writes them back in (y, v) order. */
int64_t oracle_sort_by_y(const int32_t* v, const int32_t* y, int64_t n,
                         int32_t* out_y, int32_t* out_v) {
    int64_t m = 0;
    pair32* t = sorted_by_y(v, y, n, &m);
    if (!t) return -1;
    for (int64_t i = 0; i < m; ++i) { out_y[i] = t[i].k0; out_v[i] = t[i].k1; }
    free(t);
    return m;
}
