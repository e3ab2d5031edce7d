/*
 * paper_method.c -- the paper's own CPU method for S = sparse(i,j,s,m,n),
 * written from its description (the threaded form of §3; one thread is the
 * serial method).
 *
 * TEST AND BASELINE INFRASTRUCTURE.  Used by the test suite (a third
 * cross-check of irank / jcS / irS / prS against the sort-based oracle) and
 * by the benchmark's CPU leg (the paper's method timed on the host cores).
 * The GPU library shares no code with it and never calls it.
 *
 * Source: S. Engblom and D. Lukarski, "Fast Matlab compatible sparse assembly
 * on multicore computers" (arXiv:1406.1066).
 *
 * The method (§2.3, Parts 1-4, and the App. A post-processing) orders the
 * triplets by row with a counting pass, recognises repeated (row, column)
 * pairs with a per-column record of the last row seen, numbers the unique
 * pairs column by column, and folds the values in ascending k.  It is
 * written here only in its multithreaded form (§3); run on one thread it is
 * the serial method.
 *
 * Multithreaded form (§3): the input is cut into one contiguous slice per thread;
 * each thread counts its rows privately, and per-row prefix sums over the
 * threads give every thread its own starting cursor inside each row, so
 * rank stays stable in k.  Rows are then cut into one contiguous range per
 * thread; each thread sweeps its rows with a private column cache and private
 * column counters, producing the permuted map irankP[i] = slot of the
 * triplet at rank position i.  Per-column prefix sums over the threads turn
 * the private counters into each thread's offset inside every column, and
 * the post-processing runs over the same row ranges.  Every slot belongs to
 * one row and hence to one thread, which visits its triplets in ascending k,
 * so the sums equal the serial ones bit for bit.
 *
 * Compiled with -fopenmp when the compiler supports it; otherwise the
 * pragmas are ignored and the threaded routine runs on one thread.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads the threaded routine can use (1 without OpenMP). */
int paper_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * The method on `nthreads` threads (<= 0: all available; 1: the serial
 * method).  ii, jj unit-offset int32[len], already validated against M, N.
 * Outputs irank[len] (may be NULL), jcS[N+1], irS[>= nnz], prS[>= nnz]
 * (prS may be NULL when sr is NULL).  irank_out, when not NULL, receives
 * irank[k] = irankP[i] for k = rank[i].  *threads_used (may be NULL)
 * receives the thread count actually used.  Returns nnz, or -1 when memory
 * runs out.
 */
int64_t paper_sparse_omp(const int32_t *ii, const int32_t *jj, const double *sr, int64_t len,
                         int32_t M, int32_t N, int nthreads, int32_t *irank_out, int32_t *jcS,
                         int32_t *irS, double *prS, int *threads_used) {
    int T = nthreads > 0 ? nthreads : paper_max_threads();
#ifndef _OPENMP
    T = 1;
#endif
    if (threads_used) *threads_used = T;
    /* rowcur[t][r]: thread t's cursor in row r (unit offset r = 1..M). */
    int64_t *rowcur = (int64_t *)calloc((size_t)T * ((size_t)M + 1), sizeof(int64_t));
    int64_t *rowend = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));   /* end of row r */
    int64_t *colcnt = (int64_t *)calloc((size_t)T * ((size_t)N + 1), sizeof(int64_t));
    int64_t *rank = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
    int32_t *irankP = (int32_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int32_t));
    int32_t *hcol_all = (int32_t *)calloc((size_t)T * ((size_t)N + 1), sizeof(int32_t));
    if (!rowcur || !rowend || !colcnt || !rank || !irankP || !hcol_all) {
        free(rowcur); free(rowend); free(colcnt); free(rank); free(irankP); free(hcol_all);
        return -1;
    }
    int64_t nnz = 0;
#pragma omp parallel num_threads(T)
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#else
        const int t = 0;
#endif
        int64_t *mycur = rowcur + (size_t)t * ((size_t)M + 1);
        const int64_t k0 = len * t / T, k1 = len * (t + 1) / T;
        /* Part 1: private row counts over this thread's input slice. */
        for (int64_t k = k0; k < k1; k++) mycur[ii[k]]++;
#pragma omp barrier
        /* Per row, in parallel: each thread's offset inside the row (the
           threads before it come first: input order, so rank stays stable)
           and the row's total; then the serial prefix over rows only (the
           one strictly serial step, length M); then the row starts added. */
#pragma omp for schedule(static)
        for (int32_t r = 1; r <= M; r++) {
            int64_t run = 0;
            for (int u = 0; u < T; u++) {
                int64_t *c = rowcur + (size_t)u * ((size_t)M + 1) + r;
                const int64_t cnt = *c;
                *c = run;
                run += cnt;
            }
            rowend[r] = run;
        }
#pragma omp single
        {
            for (int32_t r = 1; r <= M; r++) rowend[r] += rowend[r - 1];
        }
#pragma omp for schedule(static)
        for (int32_t r = 1; r <= M; r++) {
            const int64_t start = rowend[r - 1];
            for (int u = 0; u < T; u++) rowcur[(size_t)u * ((size_t)M + 1) + r] += start;
        }
        /* Part 2: place this slice's triplets. */
        for (int64_t k = k0; k < k1; k++) rank[mycur[ii[k]]++] = k;
#pragma omp barrier
        /* Part 3: this thread's contiguous row range, private cache/counters. */
        const int32_t r0 = (int32_t)(1 + (int64_t)M * t / T), r1 = (int32_t)((int64_t)M * (t + 1) / T);
        int32_t *hcol = hcol_all + (size_t)t * ((size_t)N + 1);
        int64_t *mycol = colcnt + (size_t)t * ((size_t)N + 1);
        const int64_t i0 = r0 > 1 ? rowend[r0 - 1] : 0;
        const int64_t i1 = r1 >= 1 ? rowend[r1] : 0;
        {
            int64_t i = i0;
            for (int32_t r = r0; r <= r1; r++) {
                for (; i < rowend[r]; i++) {
                    const int32_t c = jj[rank[i]];
                    if (hcol[c] < r) {
                        hcol[c] = r;
                        mycol[c]++;
                    }
                    irankP[i] = (int32_t)(mycol[c] - 1);
                }
            }
        }
#pragma omp barrier
        /* Part 4: per column, thread u's slots follow those of threads < u
           (their rows are smaller); the same three steps as for the rows. */
#pragma omp for schedule(static)
        for (int32_t c = 1; c <= N; c++) {
            int64_t run = 0;
            for (int u = 0; u < T; u++) {
                int64_t *p = colcnt + (size_t)u * ((size_t)N + 1) + c;
                const int64_t cnt = *p;
                *p = run;
                run += cnt;
            }
            jcS[c] = (int32_t)run;
        }
#pragma omp single
        {
            jcS[0] = 0;
            for (int32_t c = 1; c <= N; c++) jcS[c] += jcS[c - 1];
            nnz = jcS[N];
        }
#pragma omp for schedule(static)
        for (int32_t c = 1; c <= N; c++) {
            const int64_t start = jcS[c - 1];
            for (int u = 0; u < T; u++) colcnt[(size_t)u * ((size_t)N + 1) + c] += start;
        }
        for (int64_t i = i0; i < i1; i++) irankP[i] += (int32_t)mycol[jj[rank[i]]];
        /* Post-processing over the same rows: each slot's triplets are in
           one row, visited in ascending k. */
        for (int64_t i = i0; i < i1; i++) {
            irS[irankP[i]] = 0;
            if (prS) prS[irankP[i]] = 0.0;
        }
        for (int64_t i = i0; i < i1; i++) {
            const int64_t k = rank[i];
            irS[irankP[i]] = ii[k] - 1;
            if (prS && sr) prS[irankP[i]] += sr[k];
        }
        if (irank_out)
            for (int64_t i = i0; i < i1; i++) irank_out[rank[i]] = irankP[i];
    }
    free(rowcur); free(rowend); free(colcnt); free(rank); free(irankP); free(hcol_all);
    return nnz;
}
