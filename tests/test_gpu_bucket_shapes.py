"""Every shape of the column-bucket kernel, and bucket narrowing, against the
oracle.  Inputs with exactly c triplets per column make the bucket sizes
known: the width rule puts 2^cs columns in a bucket with c * 2^cs in
(target / 2, target], so the largest bucket lands in a chosen capacity class
(4096 -> 256 x 16, 6144 -> 512 x 12, 8192 -> 512 x 16).  Strategy 2 counts a
bucket's keys in a bitmap when its (column, row rank) space fits 2^16 bits,
strategy 3 always takes the radix passes."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, config, gpu_assemble
from paper_1406_1066_gb300 import fsparse

pytestmark = pytest.mark.gpu


def per_column(n_cols, c, m, seed, used_cols=None):
    g = np.random.Generator(np.random.PCG64(seed))
    cols = np.arange(1, (used_cols or n_cols) + 1, dtype=np.int32)
    jj = np.repeat(cols, c)
    g.shuffle(jj)
    ii = g.integers(1, m + 1, jj.size, dtype=np.int32)
    s = g.standard_normal(jj.size)
    return ii, jj, s


@pytest.mark.parametrize("strategy", [2, 3])
@pytest.mark.parametrize("c,target", [(32, 4096), (40, 8192), (100, 8192)],
                         ids=["bucket_4096_256x16", "bucket_5120_512x12", "bucket_6400_512x16"])
def test_bucket_shape(c, target, strategy):
    n, m = 1 << 14, 5000
    ii, jj, s = per_column(n, c, m, 61 + c)
    with config(strategy=strategy, bucket_target=target):
        g = gpu_assemble(ii, jj, s, m, n)
    assert_same(g, oracle.assemble(ii, jj, s, m, n))


@pytest.mark.parametrize("strategy", [2, 3])
def test_uneven_columns_narrow_the_buckets(strategy):
    """Half the columns empty: the average suggests 6400 per bucket, the real
    largest is 12800, so the buckets are halved before the scatter."""
    n, m = 1 << 14, 5000
    ii, jj, s = per_column(n, 100, m, 62, used_cols=n // 2)
    with config(strategy=strategy, bucket_target=8192):
        g = gpu_assemble(ii, jj, s, m, n)
    assert_same(g, oracle.assemble(ii, jj, s, m, n))


def test_three_pass_rows_without_stash_room():
    """2^19 columns x 40, rows in [1, 60000]: 5120 per bucket, ~13 bits of row
    ranks -> three sort passes, and k needs 25 bits, so the row offset does
    not fit above the digits and rows are recovered from the rank bitmap."""
    n, m = 1 << 19, 60000
    ii, jj, s = per_column(n, 40, m, 63)
    with config(strategy=2, bucket_target=8192):
        g = gpu_assemble(ii, jj, s, m, n)
    assert_same(g, oracle.assemble(ii, jj, s, m, n))


@pytest.mark.parametrize("m", [1024, 1100, 600])
def test_key_bitmap_capacity(m):
    """64 columns x 100 triplets per bucket with rows drawn from [1, m]: every
    bucket sees about min(m, 6400) distinct rows, so its key space is 64 * 1024
    = 2^16 bits exactly (bitmap), 64 * ~1100 (radix passes) or 64 * 600
    (bitmap, with many repeated (i,j) pairs).  Each bucket decides for itself."""
    n = 1 << 14
    ii, jj, s = per_column(n, 100, m, 64 + m)
    with config(strategy=2, bucket_target=8192):
        g = gpu_assemble(ii, jj, s, m, n)
    assert_same(g, oracle.assemble(ii, jj, s, m, n))


@pytest.mark.parametrize("strategy", [2, 3])
def test_bucket_ranges_in_two_passes(strategy):
    """2^21 + 2^18 columns x 16 triplets with a 1024-triplet bucket target:
    64 columns per bucket, 36864 buckets -- more than one shared-memory
    table holds, so the count and the scatter each run once per range of
    32768 buckets, every pass skipping the other range's triplets."""
    n, m = (1 << 21) + (1 << 18), 3000
    ii, jj, s = per_column(n, 16, m, 65)
    with config(strategy=strategy, bucket_target=1024):
        g = gpu_assemble(ii, jj, s, m, n)
    assert_same(g, oracle.assemble(ii, jj, s, m, n))


def exact_runs(P, r, m, n, seed):
    """P distinct (i, j) pairs, each exactly r times, shuffled."""
    g = np.random.Generator(np.random.PCG64(seed))
    keys = np.unique(g.integers(0, m * n, 2 * P, dtype=np.int64))[:P]
    idx = np.repeat(np.arange(keys.size), r)
    g.shuffle(idx)
    ii = (keys[idx] % m + 1).astype(np.int32)
    jj = (keys[idx] // m + 1).astype(np.int32)
    return ii, jj, g.standard_normal(idx.size)


@pytest.mark.parametrize("strategy", [2, 3])
@pytest.mark.parametrize("r,bucket_path", [(300, True), (384, True), (385, False)])
def test_long_runs_ranked_in_the_bucket_or_handed_over(monkeypatch, strategy, r, bucket_path):
    """Runs of up to 384 triplets are put into ascending k inside the bucket
    kernel; a longer one hands the whole call to the onesweep sort (its digit
    passes then show in the phase timings).  Exact either way."""
    m = n = 3000
    ii, jj, s = exact_runs(400, r, m, n, 90 + r)
    with config(strategy=strategy):
        monkeypatch.setenv("FSPARSE_TIMING", "1")
        g = gpu_assemble(ii, jj, s, m, n)
        names = [p for p, _ in fsparse.fsparse_last_timings()]
        monkeypatch.delenv("FSPARSE_TIMING")
    assert_same(g, oracle.assemble(ii, jj, s, m, n))
    assert "bucket_emit" in names
    assert ("digit_passes" in names) == (not bucket_path), names
