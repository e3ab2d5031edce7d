/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for Matlab-compatible
 * sparse assembly  S = sparse(i, j, s, m, n, nzmax).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The GPU library shares no
 * code, header, table or helper with it, and never calls it.
 *
 * Source: S. Engblom and D. Lukarski, "Fast Matlab compatible sparse assembly
 * on multicore computers" (arXiv:1406.1066).
 *
 *   * §1: S(i_k, j_k) = s_k, and repeated index pairs are summed.
 *   * §2.1, Eq. (2.1) and the CCS arrays below it: prS holds the values
 *     column by column, irS the zero-offset row indices, jcS the column
 *     pointer with jcS[0] = 0 and jcS[N] = nnz.  Rows ascend inside each
 *     column (the printed example and the row-wise sweep of Part 3).
 *   * §2.2, Eqs. (2.2)-(2.3): irank[k] is the final CCS slot of triplet k,
 *     irS[irank[k]] = ii[k] - 1, prS[j] sums every sr[k] with irank[k] = j,
 *     and nnz = 1 + max irank.
 *   * §2.2: the dimensions may be implicit, the largest row and column
 *     index; App. A pre-processing rejects any index below 1.
 *   * App. A post-processing: the sum runs over k in ascending order into a
 *     zero-initialised prS, i.e. the fold (((+0.0 + s_a) + s_b) + ...).
 *   * App. A pre-processing of Matlab's double index arrays (oracle_getix):
 *     a value below 1.0, or one that differs from its ceiling, is a bad
 *     index; the rest become int.  Reading for values the paper's int cannot
 *     hold: above 2^31 - 1 is a bad index too.
 *
 * The method reaches an exactly defined result, so this oracle is that
 * definition written out: sort the tuples (j, i, k) lexicographically with
 * the C library's qsort, then sweep them once.  It is NOT the paper's
 * counting algorithm (Parts 1-4 of §2.3); an independent restatement of
 * that lives in oracle/paper_parts.py.
 *
 * A planted-mistake switch (oracle_set_mutation) exists so the tests can
 * show that every pin catches a plausible bug in this file.  It is zero by
 * default and nothing outside tests/ sets it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_INDEX 2
#define ORACLE_ERR_NOMEM 5

static int g_mutation = 0;

/* Tests only: select a deliberately wrong variant (0 = the correct oracle). */
int oracle_set_mutation(int m) {
    int old = g_mutation;
    g_mutation = m;
    return old;
}

/*
 * Validation and implicit dimensions (§2.2 text before the input listing;
 * App. A pre-processing).  Every index must be >= 1; an explicit positive
 * dimension must bound its indices; a zero dimension is inferred as the
 * largest index (0 when len == 0).
 */
/*
 * App. A pre-processing: Matlab passes index arrays as double.  Each value
 * must be at least 1.0 and equal to its ceiling (an integer); NaN fails the
 * second test.  Values above 2^31 - 1 do not fit the paper's int and are bad
 * as well.  Writes the converted indices to out[len] and returns the number
 * of bad values (0 = all good; out is then complete).
 */
int64_t oracle_getix(const double *ival, int64_t len, int32_t *out) {
    int64_t bad = 0;
    for (int64_t k = 0; k < len; k++) {
        const double x = ival[k];
        int ok = !(x < 1.0 || x != ceil(x)) && x <= 2147483647.0;
        if (g_mutation == 10) ok = x >= 1.0 && x <= 2147483647.0;          /* planted: fractions accepted */
        if (g_mutation == 11) ok = !(x < 0.0 || x != ceil(x)) && x <= 2147483647.0; /* planted: zero accepted */
        if (!ok) {
            bad++;
            out[k] = 0;
        } else {
            out[k] = (int32_t)x;
        }
    }
    return bad;
}

int oracle_dims(const int32_t *ii, const int32_t *jj, int64_t len,
                int32_t m, int32_t n, int32_t *m_out, int32_t *n_out) {
    if (len < 0 || m < 0 || n < 0) return ORACLE_ERR_ARG;
    if (len > 0 && (!ii || !jj)) return ORACLE_ERR_ARG;
    int32_t mi = 0, mj = 0;
    for (int64_t k = 0; k < len; k++) {
        if (ii[k] < 1 || jj[k] < 1) return ORACLE_ERR_INDEX;
        if (ii[k] > mi) mi = ii[k];
        if (jj[k] > mj) mj = jj[k];
    }
    if (m > 0 && mi > m) return ORACLE_ERR_INDEX;
    if (n > 0 && mj > n) return ORACLE_ERR_INDEX;
    *m_out = m > 0 ? m : mi;
    *n_out = n > 0 ? n : mj;
    return ORACLE_OK;
}

typedef struct {
    int32_t col; /* j_k, unit offset */
    int32_t row; /* i_k, unit offset */
    int64_t k;   /* position in the input */
} triplet_ref;

static int by_col_row_k(const void *pa, const void *pb) {
    const triplet_ref *a = (const triplet_ref *)pa, *b = (const triplet_ref *)pb;
    if (a->col != b->col) return a->col < b->col ? -1 : 1;
    if (a->row != b->row) {
        int less = a->row < b->row;
        if (g_mutation == 4) less = !less; /* planted: rows descending */
        return less ? -1 : 1;
    }
    if (a->k != b->k) {
        int less = a->k < b->k;
        if (g_mutation == 3) less = !less; /* planted: k descending */
        return less ? -1 : 1;
    }
    return 0;
}

/*
 * Full assembly by definition.  Inputs are unit-offset (§2.2, input
 * listing); m and n must already be resolved by oracle_dims.  Outputs:
 *   irank[len], jcS[n+1], irS[>= nnz], prS[>= nnz] (prS may be NULL when
 *   sr is NULL: symbolic only).
 * Returns nnz, or -1 when memory runs out.
 */
int64_t oracle_assemble(const int32_t *ii, const int32_t *jj, const double *sr,
                        int64_t len, int32_t m, int32_t n,
                        int32_t *irank, int32_t *jcS, int32_t *irS, double *prS) {
    (void)m;
    const int transposed = (g_mutation == 6); /* planted: rows and columns swapped */
    triplet_ref *t = (triplet_ref *)malloc((size_t)(len > 0 ? len : 1) * sizeof(triplet_ref));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 2, sizeof(int64_t));
    if (!t || !cnt) {
        free(t);
        free(cnt);
        return -1;
    }
    for (int64_t k = 0; k < len; k++) {
        t[k].col = transposed ? ii[k] : jj[k];
        t[k].row = transposed ? jj[k] : ii[k];
        t[k].k = k;
    }
    qsort(t, (size_t)len, sizeof(triplet_ref), by_col_row_k);

    /* One sweep in (col, row, k) order: a new slot opens whenever (col, row)
       differs from the previous tuple; ascending k inside a slot is the
       order of the paper's post-processing insert. */
    int64_t slot = -1;
    for (int64_t p = 0; p < len; p++) {
        int fresh = (p == 0) || t[p].col != t[p - 1].col || t[p].row != t[p - 1].row;
        if (g_mutation == 8 && p > 0 && t[p].k != t[p - 1].k + 1) fresh = 1; /* planted: merge only neighbours in k */
        if (fresh) {
            slot++;
            irS[slot] = t[p].row - (g_mutation == 1 ? 0 : 1); /* planted 1: forgot zero offset */
            if (t[p].col <= n && g_mutation != 5) cnt[t[p].col]++;
            if (prS) {
                if (g_mutation == 2)
                    prS[slot] = sr[t[p].k]; /* planted: fold seeded with first term */
                else
                    prS[slot] = 0.0; /* +0.0: the insert adds into zeroed storage */
            }
        }
        if (g_mutation == 5 && t[p].col <= n) cnt[t[p].col]++; /* planted: jcS counts duplicates */
        int64_t target = slot;
        if (g_mutation == 9 && fresh && slot > 0) target = slot - 1; /* planted: heads point one slot back */
        irank[t[p].k] = (int32_t)target;
        if (prS) {
            int skip = (g_mutation == 2 && fresh);
            int last_of_run = (p + 1 == len) || t[p + 1].col != t[p].col || t[p + 1].row != t[p].row;
            if (g_mutation == 7 && last_of_run && !fresh) skip = 1; /* planted: dropped last term */
            if (!skip) prS[slot] += sr[t[p].k];
        }
    }
    int64_t nnz = slot + 1;

    /* Column pointer: exclusive prefix of the unique count per column. */
    jcS[0] = 0;
    for (int32_t c = 1; c <= n; c++) jcS[c] = (int32_t)(jcS[c - 1] + cnt[c]);
    free(t);
    free(cnt);
    return nnz;
}

/*
 * Numeric assembly through a given irank (App. A post-processing):
 * prS starts at +0.0 and receives sr[k] for k = 0, 1, ..., len-1.
 */
void oracle_numeric(const int32_t *irank, const double *sr, int64_t len,
                    int64_t nnz, double *prS) {
    for (int64_t s = 0; s < nnz; s++) prS[s] = 0.0;
    for (int64_t k = 0; k < len; k++) prS[irank[k]] += sr[k];
}

/* Adjoint of the numeric map (linear in sr, Eq. (2.3)): ds[k] = dprS[irank[k]]. */
void oracle_adjoint(const int32_t *irank, const double *dprS, int64_t len, double *ds) {
    for (int64_t k = 0; k < len; k++) ds[k] = dprS[irank[k]];
}
