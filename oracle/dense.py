"""Second, independent oracle for tiny inputs: dense brute-force accumulation.

TEST INFRASTRUCTURE (same rule as the rest of ``oracle/``).

It follows §1 of Engblom & Lukarski literally: start from an all-zero m-by-n
matrix, add s_k into entry (i_k, j_k) for k = 0, 1, ..., L-1, remember
which entries were touched, and read the touched entries out column by
column, rows ascending (the CCS layout of §2.1).  irank[k] is the position
of entry (i_k, j_k) in that read-out (Eq. (2.2)).  Pure Python loops and
Python floats (IEEE binary64), so only for m*n and L in the low thousands.
"""
from __future__ import annotations


def assemble_dense(ii, jj, s, m: int, n: int):
    """Return (irank, jcS, irS, prS) as Python lists; i, j are unit-offset."""
    L = len(ii)
    acc = [[0.0] * n for _ in range(m)]
    touched = [[False] * n for _ in range(m)]
    for k in range(L):
        r, c = int(ii[k]) - 1, int(jj[k]) - 1
        acc[r][c] = acc[r][c] + float(s[k])
        touched[r][c] = True
    where = {}
    irS, prS, jcS = [], [], [0]
    for c in range(n):
        for r in range(m):
            if touched[r][c]:
                where[(r, c)] = len(irS)
                irS.append(r)
                prS.append(acc[r][c])
        jcS.append(len(irS))
    irank = [where[(int(ii[k]) - 1, int(jj[k]) - 1)] for k in range(L)]
    return irank, jcS, irS, prS
