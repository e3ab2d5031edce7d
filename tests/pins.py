"""Pins for the CPU oracle: facts fixed by the paper or by mathematics.

Each ``pin_*`` function raises AssertionError when the oracle disagrees
with the fact it states.  ``test_oracle_pins.py`` runs them against the
oracle; ``test_oracle_mutations.py`` plants plausible mistakes in the
oracle and checks that at least one pin fails for each.
"""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
from oracle.dense import assemble_dense
from oracle.paper_parts import counting_assembly, insert
from paper_1406_1066_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_examples.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def bits(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def check_invariants(r: oracle.Result, ii, jj):
    """Structural facts every CCS result must satisfy (§2.1, §2.2)."""
    ii, jj = np.asarray(ii), np.asarray(jj)
    nnz, jcS, irS, irank = r.nnz, r.jcS, r.irS[: r.nnz], r.irank
    assert jcS[0] == 0 and jcS[-1] == nnz, "jcS[0] = 0 and jcS[n] = nnz"
    assert np.all(np.diff(jcS) >= 0), "jcS non-decreasing"
    if ii.size:
        assert nnz == 1 + int(irank.max()), "nnz = 1 + max irank (Eq. 2.2)"
        assert np.array_equal(irS[irank], ii - 1), "irS[irank[k]] = ii[k] - 1 (Eq. 2.2)"
        col_of_slot = np.searchsorted(jcS, np.arange(nnz), side="right") - 1
        assert np.array_equal(col_of_slot[irank], jj - 1), "slot irank[k] lies in column jj[k]"
        assert np.unique(irank).size == nnz, "every slot is hit"
    else:
        assert nnz == 0
    for c in range(len(jcS) - 1):
        seg = irS[jcS[c]: jcS[c + 1]]
        assert np.all(np.diff(seg) > 0), "rows strictly ascending inside a column"


# ---------------------------------------------------------------- paper values
def pin_eq21_from_sorted_input():
    g = golden()
    t = g["sorted_input"]
    r = oracle.assemble(t["ii"], t["jj"], t["s"])
    e = g["matrix_eq_2_1"]
    assert r.status == oracle.OK and (r.m, r.n) == (4, 4)
    assert r.irS.tolist() == e["irS"], "irS of Eq. (2.1)"
    assert r.jcS.tolist() == e["jcS"], "jcS of Eq. (2.1)"
    assert r.prS.tolist() == e["prS"], "prS of Eq. (2.1)"


def pin_running_example():
    g = golden()
    t = g["running_example"]
    r = oracle.assemble(t["ii"], t["jj"], t["s"])
    e = g["matrix_eq_2_1"]
    assert r.status == oracle.OK and r.nnz == g["counts_eq_2_1"]["nnz"]
    assert r.irank.tolist() == g["part4"]["irank"], "final irank, §2.3.4 example"
    assert r.jcS.tolist() == g["part4"]["jcS"], "final jcS, §2.3.4 example"
    assert r.irS.tolist() == e["irS"] and r.prS.tolist() == e["prS"], "same S as Eq. (2.1)"
    JJ = [0] * r.nnz
    for k, slot in enumerate(r.irank):
        JJ[slot] = t["jj"][k]
    assert JJ == g["part4"]["JJ"], "JJ[irank[i]] = jj[i], §2.3.4 example"
    dense = np.zeros((4, 4))
    for c in range(4):
        for p in range(r.jcS[c], r.jcS[c + 1]):
            dense[r.irS[p], c] = r.prS[p]
    assert dense.tolist() == e["dense"], "dense S of Eq. (2.1)"


# ---------------------------------------------------------------- brute force
def pin_dense_bruteforce(cases: int = 400, seed: int = 11):
    """Oracle == dense accumulation (§1 taken literally) on tiny random inputs."""
    g = np.random.Generator(np.random.PCG64(seed))
    for c in range(cases):
        m, n = int(g.integers(1, 33)), int(g.integers(1, 33))
        L = int(g.integers(0, 200))
        kind = ("normal", "int", "ones")[c % 3]
        t = inputs.random_small(L, m, n, seed * 100000 + c, dup=float(g.random()), values=kind)
        if c % 7 == 0 and L:
            t.s[g.integers(0, L, max(1, L // 4))] = -0.0
        r = oracle.assemble(t.ii, t.jj, t.s, m, n)
        assert r.status == oracle.OK
        irank, jcS, irS, prS = assemble_dense(t.ii, t.jj, t.s, m, n)
        assert r.irank.tolist() == irank, f"irank vs dense, case {c}"
        assert r.jcS.tolist() == jcS, f"jcS vs dense, case {c}"
        assert r.irS.tolist() == irS, f"irS vs dense, case {c}"
        assert np.array_equal(bits(r.prS), bits(prS)), f"prS bits vs dense, case {c}"


def pin_library_unique(seed: int = 5):
    """Order-free pins through numpy's own sort/unique on medium inputs.

    Unique (col, row) keys in ascending order are the CCS slots; their
    counts are prS when s = ones (the paper's generator uses ones, §4.2),
    and irank is the key's position among them.
    """
    for c, (L, m, n) in enumerate([(5000, 97, 89), (20000, 1000, 3), (20000, 3, 1000),
                                   (30000, 5000, 5000), (1, 7, 9)]):
        t = inputs.random_small(L, m, n, seed + c, dup=0.5, values="ones")
        r = oracle.assemble(t.ii, t.jj, t.s, m, n)
        key = (t.jj.astype(np.int64) - 1) * m + (t.ii.astype(np.int64) - 1)
        uniq, counts = np.unique(key, return_counts=True)
        assert r.nnz == uniq.size, "nnz = number of distinct pairs"
        assert np.array_equal(r.irS, (uniq % m).astype(np.int32)), "irS = rows of sorted unique keys"
        jc = np.concatenate([[0], np.cumsum(np.bincount(uniq // m, minlength=n))])
        assert np.array_equal(r.jcS, jc), "jcS = prefix of unique counts per column"
        assert np.array_equal(r.irank, np.searchsorted(uniq, key)), "irank = rank of the key"
        assert np.array_equal(r.prS, counts.astype(np.float64)), "s = ones gives multiplicities"
        check_invariants(r, t.ii, t.jj)


def pin_invariants(seed: int = 7):
    for c, (L, m, n) in enumerate([(1000, 50, 60), (4000, 7, 300), (1, 1, 1), (0, 3, 4),
                                   (2500, 1, 1), (3000, 2000, 1)]):
        t = inputs.random_small(L, m, n, seed + c, dup=0.4)
        r = oracle.assemble(t.ii, t.jj, t.s, m, n)
        assert r.status == oracle.OK
        check_invariants(r, t.ii, t.jj)


# ---------------------------------------------------------------- closed forms
def mesh_nnz(N: int, dim: int) -> int:
    """P1 mesh pattern: one diagonal per vertex, two entries per edge (§1)."""
    if dim == 2:
        V, E = N * N, 2 * N * (N - 1) + (N - 1) ** 2
    else:
        V = N ** 3
        E = 3 * N * N * (N - 1) + 3 * N * (N - 1) ** 2 + (N - 1) ** 3
    return V + 2 * E


def pin_mesh_closed_form():
    for N in (2, 3, 5, 8, 17, 64):
        t = inputs.mesh2d(N, 1)
        r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
        assert r.nnz == mesh_nnz(N, 2), f"2D nnz = V + 2E at N={N}"
        check_invariants(r, t.ii, t.jj)
    for N in (2, 3, 4, 7, 12):
        t = inputs.mesh3d(N, 2)
        r = oracle.assemble(t.ii, t.jj, t.s, t.m, t.n)
        assert r.nnz == mesh_nnz(N, 3), f"3D nnz = V + 2E at N={N}"
        check_invariants(r, t.ii, t.jj)
        # Symmetric pattern: jcS equals the row pointer of the same pattern.
        rt = oracle.assemble(t.jj, t.ii, None, t.n, t.m)
        assert np.array_equal(rt.jcS, r.jcS) and np.array_equal(rt.irS, r.irS)


# ---------------------------------------------------------------- special cases
def pin_permutation_invariance(seed: int = 3):
    t = inputs.random_small(3000, 40, 40, seed, dup=0.6, values="int")
    r = oracle.assemble(t.ii, t.jj, t.s, 40, 40)
    p = np.random.Generator(np.random.PCG64(seed)).permutation(t.L)
    rp = oracle.assemble(t.ii[p], t.jj[p], t.s[p], 40, 40)
    assert np.array_equal(r.jcS, rp.jcS) and np.array_equal(r.irS, rp.irS)
    assert np.array_equal(rp.irank, r.irank[p]), "irank permutes with the triplets"
    assert np.array_equal(r.prS, rp.prS), "small-integer sums are order-free"


def pin_runs_and_zeros():
    # Runs of length 1: prS = s, except that -0.0 becomes +0.0 (fold from +0.0).
    r = oracle.assemble([1, 2, 3], [1, 1, 2], [-0.0, 2.5, -0.0], 3, 2)
    assert bits(r.prS).tolist() == bits([0.0, 2.5, 0.0]).tolist()
    # Runs of length 2: fl(a + b).
    a, b = 0.1, 0.2
    r = oracle.assemble([2, 2], [3, 3], [a, b], 2, 3)
    assert r.nnz == 1 and bits(r.prS)[0] == bits([a + b])[0]
    assert r.jcS.tolist() == [0, 0, 0, 1] and r.irS.tolist() == [1]
    # Explicit zeros and cancelling sums keep their slot (pattern from indices only).
    r = oracle.assemble([1, 1, 2, 3], [1, 1, 1, 1], [1.0, -1.0, 0.0, 5.0], 3, 1)
    assert r.nnz == 3 and r.prS.tolist() == [0.0, 0.0, 5.0]
    # Order inside a run is ascending k: ((0 + 1) + 1e16) - 1e16 = 0, not 1.
    r = oracle.assemble([1, 1, 1], [1, 1, 1], [1.0, 1e16, -1e16], 1, 1)
    assert r.prS.tolist() == [0.0]
    r = oracle.assemble([1, 1, 1], [1, 1, 1], [-1e16, 1e16, 1.0], 1, 1)
    assert r.prS.tolist() == [1.0]
    # Non-finite values propagate as in IEEE addition.
    r = oracle.assemble([1, 1, 2, 2], [1, 1, 1, 1], [np.inf, -np.inf, np.nan, 1.0], 2, 1)
    assert np.isnan(r.prS).all()


def pin_dims_and_errors():
    r = oracle.assemble([3, 1], [2, 5], [1.0, 2.0])
    assert r.status == oracle.OK and (r.m, r.n) == (3, 5), "implicit dims = largest index (§2.2)"
    assert r.jcS.tolist() == [0, 0, 1, 1, 1, 2]
    assert oracle.assemble([0], [1], [1.0]).status == oracle.ERR_INDEX, "index below 1 (App. A)"
    assert oracle.assemble([1], [-4], [1.0]).status == oracle.ERR_INDEX
    assert oracle.assemble([4], [1], [1.0], 3, 1).status == oracle.ERR_INDEX, "row beyond m"
    assert oracle.assemble([1], [2], [1.0], 1, 1).status == oracle.ERR_INDEX, "col beyond n"
    assert oracle.assemble([1], [1], [1.0], -1, 1).status == oracle.ERR_ARG
    r = oracle.assemble([], [], [], 0, 0)
    assert r.status == oracle.OK and r.nnz == 0 and r.jcS.tolist() == [0]
    r = oracle.assemble([], [], [], 4, 6)
    assert r.status == oracle.OK and r.jcS.tolist() == [0] * 7


def pin_nzmax():
    ii, jj, s = [1, 2, 1], [1, 1, 1], [1.0, 2.0, 3.0]
    r = oracle.assemble(ii, jj, s, 2, 1, 0)
    assert r.cap == r.nnz == 2
    r = oracle.assemble(ii, jj, s, 2, 1, 5)
    assert r.nnz == 2 and r.cap == 5
    assert r.irS.tolist() == [0, 1, 0, 0, 0] and r.prS.tolist() == [4.0, 2.0, 0, 0, 0]
    assert r.jcS.tolist() == [0, 2]
    assert oracle.assemble(ii, jj, s, 2, 1, 1).status == oracle.ERR_NZMAX
    assert oracle.assemble(ii, jj, s, 2, 1, -1).status == oracle.ERR_ARG


def pin_numeric_and_adjoint(seed: int = 9):
    t = inputs.random_small(4000, 60, 50, seed, dup=0.5)
    r = oracle.assemble(t.ii, t.jj, t.s, 60, 50)
    # Numeric re-assembly through irank equals the assembled values bit for bit.
    assert np.array_equal(bits(oracle.numeric(r.irank, t.s, r.nnz)), bits(r.prS))
    # Adjoint: <dprS, A s> = <A^T dprS, s>, exact for small integers.
    g = np.random.Generator(np.random.PCG64(seed))
    si = g.integers(-5, 6, t.L).astype(np.float64)
    dp = g.integers(-5, 6, r.nnz).astype(np.float64)
    ds = oracle.adjoint(r.irank, dp)
    assert float(dp @ oracle.numeric(r.irank, si, r.nnz)) == float(ds @ si)
    # ... and A^T dprS equals the dense transpose applied to dprS.
    _, jc, ir, _ = assemble_dense(t.ii, t.jj, t.s, 60, 50)
    D = np.zeros((60, 50))
    for c in range(50):
        for p in range(jc[c], jc[c + 1]):
            D[ir[p], c] = dp[p]
    assert np.array_equal(ds, D[t.ii - 1, t.jj - 1])


def pin_paper_counting_method(seed: int = 13):
    """The paper's Parts 1-4 reproduce its printed intermediates and the oracle."""
    g = golden()
    t = g["running_example"]
    out = counting_assembly(t["ii"], t["jj"], 4, 4)
    assert out["part1_jrS"] == g["part1"]["jrS"]
    assert out["part2_rank"] == g["part2"]["rank"]
    assert out["part2_jrS"] == g["part2"]["jrS_unit_offset"]
    assert [t["ii"][k] for k in out["part2_rank"]] == g["part2"]["ii_of_rank"]
    assert out["part3_irank"] == g["part3"]["irank"]
    assert out["part3_jcS"] == g["part3"]["jcS"]
    assert out["irank"] == g["part4"]["irank"] and out["jcS"] == g["part4"]["jcS"]
    irS, prS = insert(out["irank"], t["ii"], t["s"], out["jcS"][-1])
    assert irS == g["matrix_eq_2_1"]["irS"] and prS == g["matrix_eq_2_1"]["prS"]
    rng = np.random.Generator(np.random.PCG64(seed))
    for c in range(60):
        m, n, L = int(rng.integers(1, 40)), int(rng.integers(1, 40)), int(rng.integers(0, 400))
        tt = inputs.random_small(L, m, n, seed * 1000 + c, dup=0.5)
        out = counting_assembly(tt.ii, tt.jj, m, n)
        r = oracle.assemble(tt.ii, tt.jj, tt.s, m, n)
        assert r.irank.tolist() == out["irank"] and r.jcS.tolist() == out["jcS"]
        irS, prS = insert(out["irank"], tt.ii, tt.s, r.nnz)
        assert r.irS.tolist() == irS and np.array_equal(bits(r.prS), bits(prS))


# App. A pre-processing of Matlab's double index arrays: a value below 1.0 or
# different from its ceiling is a bad index; the reading for values the
# paper's int cannot hold makes anything above 2^31 - 1 bad too.  Each case
# is (value, expected int or None for "bad"), written out by hand.
GETIX_CASES = [
    (1.0, 1), (2.0, 2), (3.0, 3), (12345.0, 12345), (2147483647.0, 2147483647),
    (0.0, None), (-0.0, None), (-1.0, None), (0.5, None), (1.5, None), (2.25, None),
    (np.nextafter(1.0, 2.0), None), (np.nextafter(2.0, 1.0), None), (5e-324, None),
    (float("nan"), None), (float("inf"), None), (float("-inf"), None),
    (2147483648.0, None), (1e300, None), (-2147483648.0, None),
]


def getix_rule(x: float):
    """The pre-processing rule restated with Python's own float predicates."""
    x = float(x)
    if np.isfinite(x) and x.is_integer() and 1 <= x <= 2**31 - 1:
        return int(x)
    return None


def pin_getix(seed: int = 21):
    vals = np.array([c[0] for c in GETIX_CASES])
    bad, out = oracle.getix(vals)
    want = [c[1] for c in GETIX_CASES]
    assert bad == sum(w is None for w in want), "bad-index count (App. A pre-processing)"
    for (x, w), o in zip(GETIX_CASES, out.tolist()):
        if w is not None:
            assert o == w, f"{x!r} converts to {w}"
    g = np.random.Generator(np.random.PCG64(seed))
    ints = g.integers(-5, 1 << 31, 4000).astype(np.float64)
    near = np.nextafter(ints, ints + g.choice([-1.0, 1.0], ints.size))
    frac = g.uniform(-3, 3e9, 4000)
    x = np.concatenate([ints, near, frac, [0.0, 1.0, 2.0**31 - 1, 2.0**31]])
    bad, out = oracle.getix(x)
    exp = [getix_rule(v) for v in x]
    assert bad == sum(e is None for e in exp)
    for v, e, o in zip(x.tolist(), exp, out.tolist()):
        if e is not None:
            assert o == e, f"{v!r} converts to {e}"
    # the running example given as Matlab doubles yields the printed Eq. (2.1) arrays
    g = golden()
    t, e = g["running_example"], g["matrix_eq_2_1"]
    r = oracle.assemble_f64(np.array(t["ii"], float), np.array(t["jj"], float), t["s"])
    assert r.status == oracle.OK and r.jcS.tolist() == e["jcS"]
    assert r.irS.tolist() == e["irS"] and r.prS.tolist() == e["prS"]
    for k, bad_value in ((4, 1.5), (0, 0.0), (12, float("nan"))):
        ii = np.array(t["ii"], float)
        ii[k] = bad_value
        assert oracle.assemble_f64(ii, np.array(t["jj"], float), t["s"]).status == oracle.ERR_INDEX

ALL_PINS = [
    pin_eq21_from_sorted_input,
    pin_running_example,
    pin_dense_bruteforce,
    pin_library_unique,
    pin_invariants,
    pin_mesh_closed_form,
    pin_permutation_invariance,
    pin_runs_and_zeros,
    pin_dims_and_errors,
    pin_nzmax,
    pin_numeric_and_adjoint,
    pin_paper_counting_method,
    pin_getix,
]
