"""The paper's own serial counting method (§2.3, Parts 1-4), restated.

TEST INFRASTRUCTURE (same rule as the rest of ``oracle/``).

Engblom & Lukarski reach the intermediate format (irank, jcS) of §2.2
without sorting, by counting:

* Part 1 (§2.3.1): count triplets per row and accumulate, giving a row
  pointer that ignores collisions (an upper bound on nnz per row).
* Part 2 (§2.3.2): place the triplet numbers row by row, stably, using that
  pointer as a moving cursor; this is the array ``rank`` and it leaves the
  cursor at the end of each row.
* Part 3 (§2.3.3): sweep the rows in order; a per-column memory of the last
  row seen detects the first occurrence of (row, col); only then the column
  count grows.  Each triplet's column-local slot is the column count minus
  one at the time it is visited.
* Part 4 (§2.3.4): accumulate the column counts into jcS and shift each
  irank by the start of its column.

This is the paper's algorithm, written from its description in Python for
small inputs.  The tests use it twice: it must reproduce every intermediate
array the paper prints for its running example, and on random inputs it
must agree with the sort-based definition in ``oracle.c``.
"""
from __future__ import annotations


def counting_assembly(ii, jj, m: int, n: int):
    """Run Parts 1-4; return a dict with the intermediates and final arrays.

    Keys: ``part1_jrS`` (length m+1), ``part2_rank`` (length L),
    ``part2_jrS`` (row ends, length m+1, the paper's unit-offset view),
    ``part3_irank``, ``part3_jcS`` (per-column unique counts, jcS[0] = 0),
    ``irank`` and ``jcS`` (final, zero-offset slots).
    """
    L = len(ii)
    rows = [int(x) for x in ii]
    cols = [int(x) for x in jj]

    # Part 1: histogram of rows, then running total; entry r ends row r.
    row_ptr = [0] * (m + 1)
    for r in rows:
        row_ptr[r] += 1
    for r in range(1, m + 1):
        row_ptr[r] += row_ptr[r - 1]
    part1 = list(row_ptr)

    # Part 2: row r starts where row r-1 ends; hand out positions in input
    # order, which keeps the placement stable.
    cursor = [0] + row_ptr[:m]          # cursor[r] = first position of row r
    rank = [0] * L
    for k in range(L):
        r = rows[k]
        rank[cursor[r]] = k
        cursor[r] += 1
    part2_ptr = cursor[1:] + [row_ptr[m]]   # ends of rows 1..m, then L

    # Part 3: row-ordered sweep with a "last row seen" memory per column.
    last_row = [0] * (n + 1)
    col_count = [0] * (n + 1)
    irank = [0] * L
    pos = 0
    for r in range(1, m + 1):
        while pos < row_ptr[r]:
            k = rank[pos]
            c = cols[k]
            if last_row[c] < r:
                last_row[c] = r
                col_count[c] += 1
            irank[k] = col_count[c] - 1
            pos += 1
    part3_irank = list(irank)
    part3_jcS = list(col_count)

    # Part 4: prefix sum over columns, then offset each slot by its column start.
    jcS = list(col_count)
    for c in range(2, n + 1):
        jcS[c] += jcS[c - 1]
    for k in range(L):
        irank[k] += jcS[cols[k] - 1]

    return {
        "part1_jrS": part1,
        "part2_rank": rank,
        "part2_jrS": part2_ptr,
        "part3_irank": part3_irank,
        "part3_jcS": part3_jcS,
        "irank": irank,
        "jcS": jcS,
    }


def insert(irank, ii, s, nnz: int):
    """App. A post-processing: irS[irank[k]] = ii[k]-1; prS[irank[k]] += s[k], k ascending."""
    irS = [0] * nnz
    prS = [0.0] * nnz
    for k in range(len(irank)):
        irS[irank[k]] = int(ii[k]) - 1
        prS[irank[k]] = prS[irank[k]] + float(s[k])
    return irS, prS
